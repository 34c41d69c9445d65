// C-ABI entry points, device storage and the level scheduler.
//
// A handle owns: the symbolic structure (host and device copies), the
// supernodal storage of the factors (`lu`), of the normalised factors
// (`nf`: Lhat and Uhat^T panels, Algorithm 1 step 2) and of the selected
// inverse (`ainv`), one scratch arena, and the launch plans.  A plan is a
// list of kernel launches whose task lists, GEMM descriptors and offsets
// live in one device arena built once per (dtype, batch); the selected-
// inversion plan can be recorded in a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "pselinv.h"

using namespace pselinv;

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return PSELINV_OK;
  if (e == cudaErrorMemoryAllocation) return PSELINV_ERR_OOM;
  return PSELINV_ERR_CUDA;
}
#define CK(x)                              \
  do {                                     \
    const cudaError_t e_ = (x);            \
    if (e_ != cudaSuccess) {               \
      (void)cudaGetLastError();            \
      return cuda_status(e_);              \
    }                                      \
  } while (0)

enum StepKind {
  ST_GEMM,
  ST_TRI_INV,
  ST_GATHER,
  ST_SCATTER_SUB,
  ST_COPY,
  ST_MEMSET,
  ST_SCATTER_VALUES,
  ST_SLICE,
  ST_OZGEMM,
  ST_ZERO,
  ST_LU_PANEL,
  ST_SMALL_LEVEL,
  ST_GSLICE,
  ST_OUTMAX,
  ST_MIRROR
};

struct Step {
  StepKind kind;
  int cfg = 0;    // GEMM: kernel config; TRI_INV: 1 small blocks; SLICE: 1 maxima pass;
                  // OZGEMM: slices; SMALL_LEVEL: shared-memory bytes of a CTA
  int n = 0;      // tasks / segments
  int n2 = 0;     // GSLICE: ordinary slice tasks after the n G tiles
  int grid = 0;
  size_t tasks = 0, descs = 0, offs = 0, offs2 = 0;  // byte offsets into the plan arena
  void* ptr = nullptr;                    // memset target / store
  void* ptr2 = nullptr;                   // second buffer
  size_t bytes = 0;
  double flops = 0;                       // useful flops of a GEMM step
  int level = -1;
  int slot = -1;      // tunable step: 0 normalisation, 1 steps 3+5, 2 step 4
  int side = 0;       // 1: side stream (normalisation, one level ahead); 2: third stream
  int wait = -1;      // event index waited on before the launch
  int signal = -1;    // event index recorded after the launch
  int param = 0;      // tuned parameter in use (GEMM tile config or K split)
  float feat[8] = {}; // shape features of the step (cost model input)
};

// events of a multi-stream plan
enum PlanEvent {
  EV_FORK = 0, EV_SIDE_JOIN = 1, EV_THIRD_JOIN = 2, EV_THIRD_DONE = 3, EV_MAIN_JOIN = 4,
  EV_THIRD_DONE2 = 5, EV_LEVEL = 6
};

struct Plan {
  std::vector<Step> steps;
  std::vector<char> host;  // staged arena
  char* arena = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool built = false;
  bool two_streams = false;
  std::vector<cudaEvent_t> ev;  // PlanEvent; EV_LEVEL + d: level d normalised

  template <class T>
  size_t push(const std::vector<T>& v) {
    size_t off = (host.size() + 255) & ~size_t(255);
    host.resize(off + v.size() * sizeof(T));
    if (!v.empty()) std::memcpy(host.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (arena) cudaFree(arena);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
    two_streams = false;
    exec = nullptr;
    graph = nullptr;
    arena = nullptr;
    steps.clear();
    host.clear();
    built = false;
  }
};

}  // namespace

struct pselinv_ctx {
  HostSym H;
  pselinv_opts opts{};
  int device = -1;
  // device structure
  void* dsym = nullptr;
  SymDev S{};
  int* derr = nullptr;
  int max_width = 1;
  // numeric state
  int dtype = 0;
  int64_t nbatch = 0;
  size_t esize = 0;
  char* lu = nullptr;
  char* nf = nullptr;
  char* ainv = nullptr;
  char* scratch = nullptr;
  size_t scratch_bytes = 0;
  size_t scratch_high = 0;  // plan building: highest scratch byte a step uses
  char* staging = nullptr;  // nbatch * nnz values
  char* outstage = nullptr; // nnz values
  // running row and column maxima of |Ainv| (nbatch * 2n bit patterns),
  // the exponents of the split sweep's G slices
  unsigned long long* rcmax = nullptr;
  // pole-expansion consumers: the input pattern (for transposed entries),
  // the storage slot of the transposed entry of every input entry, and a
  // buffer for weights, B and partial sums
  std::vector<int64_t> colptr_h, rowind_h;
  int64_t* tslot = nullptr;
  char* cbuf = nullptr;
  bool factored = false, inverted = false;
  Plan factor_plan;
  Plan selinv_plan[2][2];  // [precision][schedule]
  int slices = 6;          // FP16 slices per operand of the split products
  int last_precision = 0;
  // tuned parameters: key = (precision, level, slot) -> candidate value
  std::map<std::tuple<int, int, int>, int> tuned;
  std::vector<pselinv_tune_record> records;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t main_stream = nullptr;   // sweep launches (highest priority)
  cudaStream_t side_stream = nullptr;   // normalisation one level ahead
  cudaStream_t third_stream = nullptr;  // triangular inverses of the deeper levels (lowest)
  int64_t last_info = -1;
  int last_status = 0;
  // supernodes the selected-inversion plan covers (empty = all): one
  // rank's share of a partitioned sweep (pselinv_set_subset)
  std::vector<char> subset;
  // staging of pselinv_export_block / pselinv_import_block: tile tasks and
  // their (zero) offsets
  void* blk_buf = nullptr;
  size_t blk_buf_bytes = 0;
};

namespace {

template <class T>
int upload(std::vector<char>& host, size_t& off, const std::vector<T>& v) {
  off = (host.size() + 255) & ~size_t(255);
  host.resize(off + v.size() * sizeof(T) + 8);
  if (!v.empty()) std::memcpy(host.data() + off, v.data(), v.size() * sizeof(T));
  return 0;
}

template <class Dst, class Src>
std::vector<Dst> narrow(const std::vector<Src>& v) {
  std::vector<Dst> out(v.size());
  for (size_t i = 0; i < v.size(); i++) out[i] = (Dst)v[i];
  return out;
}

int upload_structure(pselinv_ctx* h) {
  const HostSym& H = h->H;
  std::vector<int64_t> sn_c(H.ns);
  for (int64_t k = 0; k < H.ns; k++) sn_c[k] = H.rows_ptr[k + 1] - H.rows_ptr[k];
  std::vector<char> host;
  size_t o_first, o_width, o_c, o_off, o_rptr, o_rblk, o_bsn, o_bpb, o_brel, o_rel, o_vmap;
  upload(host, o_first, narrow<int32_t>(H.sn_first));
  upload(host, o_width, narrow<int32_t>(H.sn_width));
  upload(host, o_c, narrow<int32_t>(sn_c));
  upload(host, o_off, H.sn_offset);
  upload(host, o_rptr, H.rows_ptr);
  upload(host, o_rblk, H.rows_blk);
  upload(host, o_bsn, H.blk_sn);
  upload(host, o_bpb, H.blk_pb);
  upload(host, o_brel, H.blk_rel);
  upload(host, o_rel, H.relidx);
  upload(host, o_vmap, H.value_map);
  // per-position storage bases of the gathers of G_K (fused gather and
  // slicing): the column side over R_L(K) (= R_K), the row side over R_U(K)
  size_t o_cd = 0, o_cp = 0, o_cr = 0, o_cs = 0, o_rp = 0, o_rr = 0, o_rs = 0;
  {
    auto cl = [&](int64_t J) { return H.rows_ptr[J + 1] - H.rows_ptr[J]; };
    auto cu = [&](int64_t J) {
      return H.general ? H.urows_ptr[J + 1] - H.urows_ptr[J] : cl(J);
    };
    const size_t nl = H.rows.size();
    std::vector<int64_t> cd(nl), cp(nl), cr(nl);
    std::vector<int32_t> cs(nl);
    for (int64_t k = 0; k < H.ns; k++)
      for (int64_t p = H.rows_ptr[k]; p < H.rows_ptr[k + 1]; p++) {
        const int32_t b = H.rows_blk[p];
        const int64_t J = H.blk_sn[b], sJ = H.sn_width[J], t = H.rows[p] - H.sn_first[J];
        cd[p] = H.sn_offset[J] + t * sJ;
        // Ainv(x, y), x after J: L panel of J (symmetric) or its U^T panel
        // (rows R_U(J), general)
        cp[p] = H.general ? H.sn_offset[J] + sJ * sJ + cl(J) * sJ + t * cu(J)
                          : H.sn_offset[J] + sJ * sJ + t * cl(J);
        cr[p] = H.blk_rel[b] - (H.general ? H.blk_q0[b] : H.blk_pb[b]);
        cs[p] = (int32_t)J;
      }
    const std::vector<int64_t>& uptr = H.general ? H.urows_ptr : H.rows_ptr;
    const std::vector<int64_t>& urows = H.general ? H.urows : H.rows;
    const size_t nu = urows.size();
    std::vector<int64_t> rp(nu), rr(nu);
    std::vector<int32_t> rs(nu);
    for (int64_t k = 0; k < H.ns; k++)
      for (int64_t p = uptr[k]; p < uptr[k + 1]; p++) {
        const int32_t b = H.general ? H.urows_blk[p] : H.rows_blk[p];
        const int64_t I = H.general ? H.ublk_sn[b] : H.blk_sn[b];
        const int64_t sI = H.sn_width[I], t = urows[p] - H.sn_first[I];
        // Ainv(x, y), y after I: U^T panel of I (symmetric) or its L panel
        rp[p] = H.general ? H.sn_offset[I] + sI * sI + t * cl(I)
                          : H.sn_offset[I] + sI * sI + cl(I) * sI + t * cl(I);
        rr[p] = H.general ? H.ublk_rel[b] - H.ublk_q0[b] : H.blk_rel[b] - H.blk_pb[b];
        rs[p] = (int32_t)I;
      }
    upload(host, o_cd, cd);
    upload(host, o_cp, cp);
    upload(host, o_cr, cr);
    upload(host, o_cs, cs);
    upload(host, o_rp, rp);
    upload(host, o_rr, rr);
    upload(host, o_rs, rs);
  }
  // the global index of every position of R_L(K) (R_K)
  size_t o_lrows = 0;
  upload(host, o_lrows, narrow<int32_t>(H.rows));
  // general patterns: the second row structure and its maps
  size_t o_cu = 0, o_urptr = 0, o_urows = 0, o_urblk = 0, o_q0 = 0, o_ubsn = 0, o_ubrel = 0,
         o_ubq0 = 0, o_inv = 0;
  if (H.general) {
    std::vector<int64_t> sn_cu(H.ns);
    for (int64_t k = 0; k < H.ns; k++) sn_cu[k] = H.urows_ptr[k + 1] - H.urows_ptr[k];
    upload(host, o_cu, narrow<int32_t>(sn_cu));
    upload(host, o_urptr, H.urows_ptr);
    upload(host, o_urows, narrow<int32_t>(H.urows));
    upload(host, o_urblk, H.urows_blk);
    upload(host, o_q0, H.blk_q0);
    upload(host, o_ubsn, H.ublk_sn);
    upload(host, o_ubrel, H.ublk_rel);
    upload(host, o_ubq0, H.ublk_q0);
    upload(host, o_inv, H.inv_map);
  }
  CK(cudaMalloc(&h->dsym, host.size() + 256));
  CK(cudaMemcpy(h->dsym, host.data(), host.size(), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&h->derr, 4 * sizeof(int)));
  CK(cudaMemset(h->derr, 0, 4 * sizeof(int)));
  char* b = (char*)h->dsym;
  SymDev& S = h->S;
  S.sn_first = (const int32_t*)(b + o_first);
  S.sn_width = (const int32_t*)(b + o_width);
  S.sn_c = (const int32_t*)(b + o_c);
  S.sn_off = (const int64_t*)(b + o_off);
  S.rows_ptr = (const int64_t*)(b + o_rptr);
  S.rows_blk = (const int32_t*)(b + o_rblk);
  S.blk_sn = (const int32_t*)(b + o_bsn);
  S.blk_pb = (const int32_t*)(b + o_bpb);
  S.blk_rel = (const int64_t*)(b + o_brel);
  S.relidx = (const int32_t*)(b + o_rel);
  S.value_map = (const int64_t*)(b + o_vmap);
  S.storage = H.storage;
  S.nnz = H.nnz;
  S.ns = (int32_t)H.ns;
  S.check = h->opts.check_level > 0 ? 1 : 0;
  S.relidx_size = (int64_t)H.relidx.size();
  S.err = h->derr;
  S.out_map = S.value_map;
  S.general = H.general ? 1 : 0;
  S.col_diag = (const int64_t*)(b + o_cd);
  S.col_pan = (const int64_t*)(b + o_cp);
  S.col_rel = (const int64_t*)(b + o_cr);
  S.col_sn = (const int32_t*)(b + o_cs);
  S.row_pan = (const int64_t*)(b + o_rp);
  S.row_rel = (const int64_t*)(b + o_rr);
  S.row_sn = (const int32_t*)(b + o_rs);
  S.lrows = (const int32_t*)(b + o_lrows);
  S.urows = S.lrows;
  S.n = H.n;
  if (H.general) {
    S.sn_cu = (const int32_t*)(b + o_cu);
    S.urows_ptr = (const int64_t*)(b + o_urptr);
    S.urows = (const int32_t*)(b + o_urows);
    S.urows_blk = (const int32_t*)(b + o_urblk);
    S.blk_q0 = (const int32_t*)(b + o_q0);
    S.ublk_sn = (const int32_t*)(b + o_ubsn);
    S.ublk_rel = (const int64_t*)(b + o_ubrel);
    S.ublk_q0 = (const int32_t*)(b + o_ubq0);
    S.out_map = (const int64_t*)(b + o_inv);
  }
  return PSELINV_OK;
}

inline int64_t cK(const HostSym& H, int64_t K) { return H.rows_ptr[K + 1] - H.rows_ptr[K]; }
// rows of K's U^T panel: |R_U(K)| for a general pattern, else c_K
inline int64_t cU(const HostSym& H, int64_t K) {
  return H.general ? H.urows_ptr[K + 1] - H.urows_ptr[K] : cK(H, K);
}

int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

template <class D>
void gemm_features(Step& st, const std::vector<D>& descs, double kscale);
template <>
void gemm_features<GemmDesc>(Step& st, const std::vector<GemmDesc>& descs, double);

// GEMM step from a list of descriptors; tasks enumerate every tile and K chunk
// lower_c: only the tasks of C on or below its diagonal (a symmetric
// product whose upper triangle nobody reads)
void add_gemm_step(Plan& P, int dtype, int cfg, const std::vector<GemmDesc>& descs, int level,
                   int slot = -1, bool lower_c = false) {
  if (descs.empty()) return;
  if (cfg == GEMM_ROWS)
    for (const GemmDesc& g : descs)
      if (!rows_eligible(g)) cfg = GEMM_32x32;
  std::vector<GemmTask> tasks;
  std::vector<double> work;  // GEMM_ROWS: FMAs per task, for the launch order
  double flops = 0, bytes = 0;
  for (size_t d = 0; d < descs.size(); d++) {
    const GemmDesc& g = descs[d];
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) continue;
    if (cfg == GEMM_ROWS) {
      const int tri = g.tri & (GEMM_TRI_LOWER_B | GEMM_TRI_UPPER_B);
      const int kchunk = ceil_div(g.K, g.ksplit);
      for (int tn = 0; tn < ceil_div(g.N, kRowsChunk); tn++) {
        const int j0 = tn * kRowsChunk, w = std::min(kRowsChunk, g.N - j0);
        const int nw = w <= 4 ? 4 : 8;
        for (int ks = 0; ks < g.ksplit; ks++) {
          int kb = ks * kchunk, ke = std::min(g.K, kb + kchunk);
          if (tri == GEMM_TRI_LOWER_B) kb = std::max(kb, j0);       // op(B)(k, n) = 0 for k < n
          if (tri == GEMM_TRI_UPPER_B) ke = std::min(ke, j0 + w);   // op(B)(k, n) = 0 for k > n
          if (kb >= ke) continue;
          const double kw = ke - kb;
          for (int tm = 0; tm < ceil_div(g.M, kRowsBlock); tm++) {
            if (lower_c && (tm + 1) * kRowsBlock <= j0) continue;  // above the diagonal
            tasks.push_back({(int)d, tm, tn, nw + 16 * ks});
            work.push_back(kw * nw * std::min(kRowsBlock, g.M - tm * kRowsBlock));
          }
        }
      }
    } else {
      const int bm = gemm_tile_m(dtype, cfg), bn = gemm_tile_n(dtype, cfg);
      for (int ks = 0; ks < g.ksplit; ks++)
        for (int tn = 0; tn < ceil_div(g.N, bn); tn++)
          for (int tm = 0; tm < ceil_div(g.M, bm); tm++)
            if (!lower_c || (tm + 1) * bm > tn * bn) tasks.push_back({(int)d, tm, tn, ks});
    }
    double f = 2.0 * g.M * g.N * g.K;
    if (lower_c) f = (double)g.M * (g.N + 1) * g.K;  // the lower triangle of a square C
    if (g.tri == GEMM_TRI_LOWER_B || g.tri == GEMM_TRI_UPPER_B) f = (double)g.M * g.N * (g.N + 1);
    if (g.tri == (GEMM_TRI_UPPER_A | GEMM_TRI_LOWER_B)) f = 2.0 * g.N * (double)g.N * g.N / 3.0;
    flops += f * (dtype == DT_F64 ? 1 : 4);
    const double es = dtype == DT_F64 ? 8.0 : 16.0;
    bytes += es * ((double)g.M * g.K + (double)g.K * g.N +
                   (double)g.M * g.N * ((g.atomic || g.beta != 0.0) ? 2.0 : 1.0));
  }
  if (tasks.empty()) return;
  if (cfg == GEMM_ROWS) {  // longest tasks first: CTAs start in task order
    std::vector<size_t> order(tasks.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return work[a] > work[b]; });
    std::vector<GemmTask> sorted(tasks.size());
    for (size_t i = 0; i < order.size(); i++) sorted[i] = tasks[order[i]];
    tasks.swap(sorted);
  }
  Step s;
  s.bytes = (size_t)bytes;
  s.kind = ST_GEMM;
  s.cfg = cfg;
  s.n = (int)tasks.size();
  s.grid = std::min(s.n, 1 << 20);
  s.descs = P.push(descs);
  s.tasks = P.push(tasks);
  s.flops = flops;
  s.level = level;
  s.slot = slot;
  s.param = cfg;
  gemm_features(s, descs, 0);
  P.steps.push_back(s);
}

GemmDesc make_desc(const void* A, const void* B, void* C, int M, int N, int K, int lda, int ldb,
                   int ldc, int ta, int tb, double alpha, double beta, int atomic = 0,
                   int ksplit = 1, int tri = 0) {
  GemmDesc d;
  d.tri = tri;
  d.A = A;
  d.B = B;
  d.C = C;
  d.M = M;
  d.N = N;
  d.K = K;
  d.lda = lda;
  d.ldb = ldb;
  d.ldc = ldc;
  d.transA = ta;
  d.transB = tb;
  d.alpha = alpha;
  d.beta = beta;
  d.atomic = atomic;
  d.ksplit = ksplit < 1 ? 1 : ksplit;
  return d;
}

inline int64_t r64(int64_t r) { return (r + 63) / 64; }
inline int64_t k32(int64_t k) { return (k + 31) / 32; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
inline size_t slice_bytes(int64_t R, int64_t Kd, int S) {
  return align256((size_t)S * r64(R) * k32(Kd) * 4096);
}
inline size_t exps_bytes(int64_t R) { return align256((size_t)R * 4); }

// bytes one supernode needs during a split-precision level: five slice sets
// (G by rows, G by columns, Lhat, Uhat^T, Ainv(C,K)) and their exponents (G
// itself is sliced straight from the ancestors' blocks, never stored)
size_t ozaki_sn_bytes(int64_t s, int64_t c, int S, size_t es) {
  if (c == 0) return 0;
  const size_t parts = es / 8;  // complex: real and imaginary slice halves
  return 2 * (parts * slice_bytes(c, c, S) + exps_bytes(c)) +
         3 * (parts * slice_bytes(s, c, S) + exps_bytes(s)) + (size_t)(2 * c + 3 * s) * 8 + 2048;
}
size_t ozaki_level_bytes(const HostSym& H, int64_t nb, int S, size_t es) {
  size_t mx = 0;
  for (size_t d = 0; d + 1 < H.level_ptr.size(); d++) {
    size_t b = 0;
    for (int64_t i = H.level_ptr[d]; i < H.level_ptr[d + 1]; i++) {
      const int64_t K = H.level_sn[i];
      b += ozaki_sn_bytes(H.sn_width[K], std::max(cK(H, K), cU(H, K)), S, es);
    }
    mx = std::max(mx, b * (size_t)nb);
  }
  return mx;
}

// bytes of the split normalisation of the largest level
size_t ozaki_norm_bytes(const HostSym& H, int64_t nb, int S, size_t es) {
  const size_t parts = es / 8;
  size_t mx = 0;
  for (size_t d = 0; d + 1 < H.level_ptr.size(); d++) {
    size_t b = 512;
    for (int64_t i = H.level_ptr[d]; i < H.level_ptr[d + 1]; i++) {
      const int64_t K = H.level_sn[i], s = H.sn_width[K], c = cK(H, K);
      b += 2 * (parts * slice_bytes(s, s, S) + exps_bytes(s) + 512) + (size_t)(2 * c + 2 * s) * 8;
      if (c > 0) b += 2 * (parts * slice_bytes(c, s, S) + exps_bytes(c) + 512);
    }
    mx = std::max(mx, b * (size_t)nb + 512);
  }
  return mx;
}

// scratch of the selected-inversion sweep before the normalisation region:
// W (2 s^2 for every supernode) and the largest level's G (FP64 levels) or
// split-level operands
size_t selinv_main_bytes(const HostSym& H, int64_t nb, size_t es) {
  int64_t w = 0, gmax = 0;
  for (int64_t k = 0; k < H.ns; k++) w += 2 * H.sn_width[k] * H.sn_width[k];
  for (size_t d = 0; d + 1 < H.level_ptr.size(); d++) {
    int64_t g = 0;
    for (int64_t i = H.level_ptr[d]; i < H.level_ptr[d + 1]; i++) {
      g += cK(H, H.level_sn[i]) * cU(H, H.level_sn[i]);
    }
    gmax = std::max(gmax, g);
  }
  return align256(std::max((size_t)((w + gmax) * nb) * es + 256,
                           (size_t)(w * nb) * es + ozaki_level_bytes(H, nb, 6, es) + 4096));
}

// row and column maxima of the split levels' operands, a region of their
// own for the whole sweep (zeroed once per sweep): an upper bound with one
// group per supernode
size_t maxima_bytes(const HostSym& H, int64_t nb) {
  size_t b = 0;
  for (int64_t K = 0; K < H.ns; K++)
    if (cK(H, K) > 0 || cU(H, K) > 0)
      b += align256((size_t)(cK(H, K) + cU(H, K) + 3 * H.sn_width[K]) * 8 * nb + 8);
  return b;
}

// scratch needed (bytes) by the factor and selected-inversion plans; the
// split normalisation (side stream) has its own region after the sweep's,
// the maxima theirs after that
size_t scratch_need(const HostSym& H, int64_t nb, size_t es) {
  // factorisation levels: W, the panels and the Schur product in FP64, then
  // the slices of a split level's operands (counted for every level)
  size_t fmax = 0;
  const size_t parts = es / 8;
  for (size_t d = 0; d + 1 < H.hlevel_ptr.size(); d++) {
    int64_t f = 0;
    size_t oz = 512;
    for (int64_t i = H.hlevel_ptr[d]; i < H.hlevel_ptr[d + 1]; i++) {
      const int64_t K = H.hlevel_sn[i], s = H.sn_width[K], c = cK(H, K), cu = cU(H, K);
      f += 2 * s * s + (c + cu) * s + c * cu;
      if (c > 0 && cu > 0)  // A_{C,K}, A_{K,C}^T, Uinv, Linv (the solves; then TL, TU)
        oz += parts * (slice_bytes(c, s, 6) + slice_bytes(cu, s, 6) + 2 * slice_bytes(s, s, 6)) +
              exps_bytes(c) + exps_bytes(cu) + 2 * exps_bytes(s) + 2048 +
              (size_t)(c + cu + 2 * s) * 8;
    }
    fmax = std::max(fmax, align256((size_t)(f * nb) * es) + oz * (size_t)nb + 512);
  }
  return std::max(fmax + 256,
                  selinv_main_bytes(H, nb, es) + ozaki_norm_bytes(H, nb, 6, es) +
                      maxima_bytes(H, nb));
}

// default FP64 kernel before tuning: row panels for level launches (what
// the tuner keeps for most FP64 launches of the 40^3 sweep, and faster than
// tiles on the factorisation's Schur products); 32 x 32 tiles for launches
// of one supernode's products, where more, smaller tasks fill the GPU
// better (40^3 per-supernode sweep 274 vs 318 ms)
int choose_cfg(int schedule) {
  return schedule == PSELINV_SCHED_PER_SUPERNODE ? GEMM_32x32 : GEMM_ROWS;
}

int tuned_value(const pselinv_ctx* h, int prec, int level, int slot, int dflt) {
  auto it = h->tuned.find(std::make_tuple(prec, level, slot));
  return it == h->tuned.end() ? dflt : it->second;
}

// shape features of a GEMM step (log2 scale): problem count, total flops,
// largest and mean M, N, K
template <class D>
void gemm_features(Step& st, const std::vector<D>& descs, double kscale) {
  double n = 0, fl = 0, mm = 0, mn = 0, mk = 0, sm = 0, sn = 0, sk = 0;
  for (const auto& d : descs) {
    const double K = kscale > 0 ? d.K32 * kscale : 0;
    n += 1;
    fl += 2.0 * d.M * d.N * K;
    mm = std::max(mm, (double)d.M);
    mn = std::max(mn, (double)d.N);
    mk = std::max(mk, K);
    sm += d.M;
    sn += d.N;
    sk += K;
  }
  const double v[8] = {n, fl, mm, mn, mk, n ? sm / n : 0, n ? sn / n : 0, n ? sk / n : 0};
  for (int i = 0; i < 8; i++) st.feat[i] = (float)std::log2(1.0 + v[i]);
}
template <>
void gemm_features<GemmDesc>(Step& st, const std::vector<GemmDesc>& descs, double) {
  double n = 0, fl = 0, mm = 0, mn = 0, mk = 0, sm = 0, sn = 0, sk = 0;
  for (const auto& d : descs) {
    n += 1;
    fl += 2.0 * d.M * d.N * d.K;
    mm = std::max(mm, (double)d.M);
    mn = std::max(mn, (double)d.N);
    mk = std::max(mk, (double)d.K);
    sm += d.M;
    sn += d.N;
    sk += d.K;
  }
  const double v[8] = {n, fl, mm, mn, mk, n ? sm / n : 0, n ? sn / n : 0, n ? sk / n : 0};
  for (int i = 0; i < 8; i++) st.feat[i] = (float)std::log2(1.0 + v[i]);
}

// Triangular-inverse launches over blocks {instance, supernode, W offset}:
// blocks of width <= 32 one warp per triangle (cfg 1), wider ones in panels
// of 8 columns, one warp per column (cfg 0).
struct TriBlock {
  int64_t b, K, w0;
};
void add_tri_step(Plan& P, const HostSym& H, const std::vector<TriBlock>& blocks, int level,
                  int stream, bool allow_small = true) {
  std::vector<SnTask> wide, small;
  std::vector<int64_t> wofs_wide, wofs_small;
  for (const TriBlock& t : blocks) {
    const int64_t s = H.sn_width[t.K];
    for (int which = 0; which < 2; which++) {
      if (s <= 32 && allow_small) {
        small.push_back({(int)t.b, (int)t.K, which, 0});
        wofs_small.push_back(t.w0 + which * s * s);
        continue;
      }
      for (int64_t j = 0; j < s; j += 8) {
        wide.push_back({(int)t.b, (int)t.K, which, (int)j});
        wofs_wide.push_back(t.w0 + which * s * s);
      }
    }
  }
  auto push = [&](const std::vector<SnTask>& tasks, const std::vector<int64_t>& wofs, int cfg) {
    if (tasks.empty()) return;
    Step st;
    st.kind = ST_TRI_INV;
    st.cfg = cfg;
    st.n = (int)tasks.size();
    st.tasks = P.push(tasks);
    st.offs = P.push(wofs);
    st.level = level;
    st.side = stream;
    P.steps.push_back(st);
  };
  push(wide, wofs_wide, 0);
  push(small, wofs_small, 1);
}

// ---------------------------------------------------------------------------
// factor plan: scatter A, then per height level (leaves first):
//   diagonal LU, triangular inverses, L = A_{C,K} U_KK^{-1},
//   U^T = A_{K,C}^T L_KK^{-T}, Schur Sc = L U, scatter -Sc into ancestors,
//   copy the panels back.
// ---------------------------------------------------------------------------
void add_copy_step(Plan& P, const std::vector<CopySeg>& segs, int level, size_t es);

// trailing updates of the blocked diagonal LU (K = 32): 32 x 32 tiles (row
// panels: 61.9 vs 60.9 ms for the 40^3 factorisation)
constexpr int kLuUpdateCfg = GEMM_32x32;

// one supernode's products of the factorisation: the triangular solves
// TL = AL Uinv (AL = A_{C,K}, c x s) and TU = AU Linv^T (AU = A_{K,C}^T,
// cu x s), and the Schur complement Sc = TL TU^T (c x cu, K = s); column
// major
struct SchurProduct {
  char *TL, *TU, *Sc;
  int c, cu, s;
  const char *AL, *AU, *Uinv, *Linv;
};
void add_ozaki_trsm(pselinv_ctx* h, Plan& P, const std::vector<SchurProduct>& prods, int lev,
                    size_t base);
void add_ozaki_schur(pselinv_ctx* h, Plan& P, const std::vector<SchurProduct>& prods, int lev,
                     size_t base, bool lower);

int build_factor_plan(pselinv_ctx* h) {
  const HostSym& H = h->H;
  Plan& P = h->factor_plan;
  P.release();
  h->scratch_high = 0;
  const size_t es = h->esize;
  const int dt = h->dtype;
  const int64_t nb = h->nbatch;
  Step ms;
  ms.kind = ST_MEMSET;
  ms.ptr = h->lu;
  ms.bytes = (size_t)nb * H.storage * es;
  P.steps.push_back(ms);
  Step sv;
  sv.kind = ST_SCATTER_VALUES;
  P.steps.push_back(sv);
  // symmetric values (A = A^T): U_{K,C}^T = A_{C,K} L_KK^{-T} and the Schur
  // complement is symmetric, so the updates go to the lower triangle only
  // (entries (x, y), x >= y: diagonal blocks and L panels; half the Schur
  // work) and U^T panels are solved from the L panels; each diagonal block's
  // upper triangle is mirrored from its lower one before its LU
  const bool ldlt = h->opts.symmetric != 0 && !H.general;
  for (size_t lev = 0; lev + 1 < H.hlevel_ptr.size(); lev++) {
    std::vector<SnTask> diag, gt;
    std::vector<TriBlock> tri;
    std::vector<int64_t> gofs;
    std::vector<GemmDesc> trsm, schur;
    std::vector<SchurProduct> sprods;
    std::vector<CopySeg> segs;
    int64_t off = 0;  // scalars into scratch
    for (int64_t b = 0; b < nb; b++)
      for (int64_t i = H.hlevel_ptr[lev]; i < H.hlevel_ptr[lev + 1]; i++) {
        // c: rows of the L panel (R_K, or R_L(K) for a general pattern),
        // cu: rows of the U^T panel (c, or R_U(K))
        const int64_t K = H.hlevel_sn[i], s = H.sn_width[K], c = cK(H, K), cu = cU(H, K);
        const int64_t w0 = off, t0 = w0 + 2 * s * s, s0 = t0 + (c + cu) * s;
        off = s0 + c * cu;
        diag.push_back({(int)b, (int)K, 0, 0});
        if (c == 0 && cu == 0) continue;
        tri.push_back({b, K, w0});
        char* base = h->lu + ((size_t)b * H.storage + H.sn_offset[K]) * es;
        char* Lp = base + (size_t)s * s * es;
        char* Up = Lp + (size_t)c * s * es;
        char* Linv = h->scratch + (size_t)w0 * es;
        char* Uinv = Linv + (size_t)s * s * es;
        char* TL = h->scratch + (size_t)t0 * es;
        char* TU = TL + (size_t)c * s * es;
        char* Sc = h->scratch + (size_t)s0 * es;
        // L = A U^-1, U^T = A^T L^-T: both B operands upper triangular
        if (c > 0)
          trsm.push_back(make_desc(Lp, Uinv, TL, c, s, s, c, s, c, 0, 0, 1.0, 0.0, 0, 1,
                                   GEMM_TRI_UPPER_B));
        if (cu > 0)
          trsm.push_back(make_desc(ldlt ? Lp : Up, Linv, TU, cu, s, s, cu, s, cu, 0, 1, 1.0, 0.0,
                                   0, 1, GEMM_TRI_UPPER_B));
        if (c > 0 && cu > 0) {
          schur.push_back(make_desc(TL, TU, Sc, c, cu, s, c, cu, c, 0, 1, 1.0, 0.0));
          sprods.push_back({TL, TU, Sc, (int)c, (int)cu, (int)s, Lp, ldlt ? Lp : Up, Uinv, Linv});
          for (int tq = 0; tq < ceil_div(cu, 32); tq++)
            for (int tp = ldlt ? tq : 0; tp < ceil_div(c, 32); tp++) {
              gt.push_back({(int)b, (int)K, tp, tq});
              gofs.push_back(s0);
            }
        }
        segs.push_back({TL, Lp, (c + cu) * s});
      }
    // blocked LU of the diagonal blocks: panels of 32 columns, each a panel
    // launch (pivot block, L21 rows, U12 columns) and a trailing-update GEMM,
    // batched over the level's supernodes
    int64_t smax = 0;
    for (const SnTask& t : diag) smax = std::max<int64_t>(smax, H.sn_width[t.K]);
    if (ldlt && !diag.empty()) {
      Step mr;
      mr.kind = ST_MIRROR;
      mr.n = (int)diag.size();
      mr.tasks = P.push(diag);
      mr.level = (int)lev;
      P.steps.push_back(mr);
    }
    for (int64_t j0 = 0; j0 < smax; j0 += 32) {
      std::vector<SnTask> piv, pan;
      std::vector<GemmDesc> upd;
      for (const SnTask& t : diag) {
        const int64_t s = H.sn_width[t.K];
        if (s <= j0) continue;
        const int64_t w = std::min<int64_t>(32, s - j0), rest = s - j0 - w;
        const int nbk = (int)ceil_div(rest, 32);
        piv.push_back({t.inst, t.K, (int)j0, 0});
        for (int blk = 1; blk <= 2 * nbk; blk++) pan.push_back({t.inst, t.K, (int)j0, blk});
        if (rest > 0) {
          char* D = h->lu + ((size_t)t.inst * H.storage + H.sn_offset[t.K]) * es;
          upd.push_back(make_desc(D + (size_t)(j0 + w + j0 * s) * es, D + (size_t)(j0 + (j0 + w) * s) * es,
                                  D + (size_t)((j0 + w) + (j0 + w) * s) * es, (int)rest, (int)rest,
                                  (int)w, (int)s, (int)s, (int)s, 0, 0, -1.0, 1.0));
        }
      }
      for (const auto* list : {&piv, &pan}) {
        if (list->empty()) continue;
        Step d;
        d.kind = ST_LU_PANEL;
        d.n = (int)list->size();
        d.tasks = P.push(*list);
        d.level = (int)lev;
        P.steps.push_back(d);
      }
      add_gemm_step(P, dt, kLuUpdateCfg, upd, (int)lev);
    }
    // split precision: the triangular solves and the Schur products of
    // levels with enough Schur work as sliced tensor-core products (their
    // operands sliced from the level's scratch after its FP64 region);
    // otherwise FP64 row panels, which beat 64 x 64 tiles on these products
    // at every width (40^3 factorisation 61.9 -> 57.1 ms)
    double sflops = 0;
    for (const SchurProduct& q : sprods) sflops += 2.0 * q.c * q.cu * q.s;
    const double min_flops = h->opts.factor_split_mflops < 0    ? 0.0
                             : h->opts.factor_split_mflops == 0 ? 2e8
                                                                : 1e6 * h->opts.factor_split_mflops;
    const bool split = h->opts.factor_precision == PSELINV_PREC_OZAKI_FP16 && !sprods.empty() &&
                       sflops >= min_flops;
    add_tri_step(P, H, tri, (int)lev, 0);
    if (split && sprods.size() * 2 == trsm.size()) {
      add_ozaki_trsm(h, P, sprods, (int)lev, align256((size_t)off * es));
    } else {
      add_gemm_step(P, dt, GEMM_ROWS, trsm, (int)lev);
    }
    if (split)
      add_ozaki_schur(h, P, sprods, (int)lev, align256((size_t)off * es), ldlt);
    else
      add_gemm_step(P, dt, GEMM_ROWS, schur, (int)lev, -1, ldlt);
    if (!gt.empty()) {
      Step sc;
      sc.kind = ST_SCATTER_SUB;
      sc.cfg = ldlt ? 1 : 0;
      sc.n = (int)gt.size();
      sc.tasks = P.push(gt);
      sc.offs = P.push(gofs);
      sc.level = (int)lev;
      P.steps.push_back(sc);
    }
    add_copy_step(P, segs, (int)lev, es);
  }
  if (h->scratch_high > h->scratch_bytes) return PSELINV_ERR_CHECK;
  CK(cudaMalloc(&P.arena, P.host.size() + 256));
  CK(cudaMemcpy(P.arena, P.host.data(), P.host.size(), cudaMemcpyHostToDevice));
  P.built = true;
  return PSELINV_OK;
}

// ---------------------------------------------------------------------------
// selected-inversion plan (FP64 / complex128 products):
//   normalise (all supernodes at once): Linv, Uinv; Lhat = L Linv,
//   Uhat^T = U^T Uinv^T, D = Uinv Linv (-> Ainv_KK);
//   then for every depth level (roots first): gather G = Ainv_CC,
//   Ainv_CK = -G Lhat, (Ainv_KC)^T = -G^T Uhat^T, Ainv_KK += -Uhat Ainv_CK.
// schedule = PER_SUPERNODE issues the three level launches per supernode.
// ---------------------------------------------------------------------------
void add_zero_step(Plan& P, const std::vector<CopySeg>& segs, int level) {
  if (segs.empty()) return;
  Step z;
  z.kind = ST_ZERO;
  int64_t longest = 0;
  for (const CopySeg& g : segs) longest = std::max(longest, g.count);
  z.grid = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (longest + 2047) / 2048));
  z.n = (int)segs.size();
  z.tasks = P.push(segs);
  z.level = level;
  P.steps.push_back(z);
}

void add_copy_step(Plan& P, const std::vector<CopySeg>& segs, int level, size_t es) {
  if (segs.empty()) return;
  Step cp;
  cp.kind = ST_COPY;
  cp.n = (int)segs.size();
  cp.tasks = P.push(segs);
  cp.level = level;
  double bytes = 0;
  int64_t longest = 0;
  for (const CopySeg& g : segs) {
    bytes += 2.0 * (double)g.count * (double)es;  // read + write
    longest = std::max(longest, g.count);
  }
  cp.bytes = (size_t)bytes;
  // CTAs per segment: about 8 elements per thread of the longest segment
  cp.grid = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (longest + 2047) / 2048));
  P.steps.push_back(cp);
}

void add_slice_step(Plan& P, const std::vector<SliceDesc>& descs, int level, bool maxima) {
  if (descs.empty()) return;
  std::vector<SliceTask> tasks;
  double bytes = 0;
  for (size_t d = 0; d < descs.size(); d++) {
    for (int kc = 0; kc < ceil_div(descs[d].K32, 2); kc++)
      for (int rb = 0; rb < descs[d].R64; rb++) tasks.push_back({(int)d, rb, kc});
    bytes += 8.0 * descs[d].R * descs[d].Kd;
    if (!maxima) bytes += 2.0 * descs[d].S * descs[d].R64 * 64.0 * descs[d].K32 * 32;
  }
  Step st;
  st.cfg = maxima ? 1 : 0;
  st.kind = ST_SLICE;
  st.n = (int)tasks.size();
  st.descs = P.push(descs);
  st.tasks = P.push(tasks);
  st.bytes = (size_t)bytes;
  st.level = level;
  P.steps.push_back(st);
}

// Maxima (maxima = true) or slicing pass over the G tiles of a level and
// the ordinary slice sets descs[dense[i]] of its panels, in one launch.
void add_gslice_step(Plan& P, const std::vector<SliceDesc>& descs,
                     const std::vector<GTileTask>& gtasks, const std::vector<int>& dense,
                     int level, bool maxima, size_t es) {
  if (gtasks.empty() && dense.empty()) return;
  std::vector<SliceTask> st;
  double bytes = 0;
  for (int d : dense) {
    const SliceDesc& g = descs[d];
    for (int kc = 0; kc < ceil_div(g.K32, 2); kc++)
      for (int rb = 0; rb < g.R64; rb++) st.push_back({d, rb, kc});
    bytes += 8.0 * g.R * g.Kd * (g.cplx ? 2 : 1);
    if (!maxima) bytes += 2.0 * g.S * g.R64 * 64.0 * g.K32 * 32;
  }
  for (const GTileTask& t : gtasks) {
    const SliceDesc& g = descs[t.dr];
    const double rows = std::min(64, g.R - 64 * t.tp), cols = std::min(64, g.R - 64 * t.tq);
    bytes += rows * cols * (double)es;  // the tile's entries, read once
    if (!maxima)  // its slices in one or two layouts
      bytes += (t.dc >= 0 ? 2.0 : 1.0) * 2.0 * g.S * 64.0 * 64.0 * (g.cplx ? 2 : 1);
  }
  Step s;
  s.kind = ST_GSLICE;
  s.cfg = maxima ? 1 : 0;
  s.n = (int)gtasks.size();
  s.n2 = (int)st.size();
  s.descs = P.push(descs);
  s.tasks = P.push(gtasks);
  s.offs = P.push(st);
  s.bytes = (size_t)bytes;
  s.level = level;
  P.steps.push_back(s);
}

// K blocks (of 32) of one exact accumulation chunk of the sliced GEMM, and
// the most chunks one task may add into its 64-bit totals
constexpr int kOzChunkBlocks = 16;
constexpr int kOzMaxChunks = 31;

// smallest K split keeping every task within kOzMaxChunks chunks
int min_ozaki_ksplit(const OzDesc& d) {
  return std::max(1, ceil_div(d.K32, kOzChunkBlocks * kOzMaxChunks));
}

// ksplit so that a launch has about two CTAs per SM (one CTA fits an SM)
int choose_ozaki_ksplit(const std::vector<OzDesc>& descs) {
  int64_t tiles = 0, kmax = 1;
  for (const auto& d : descs) {
    tiles += (int64_t)ceil_div(d.M, 128) * ceil_div(d.N, 64);
    kmax = std::max<int64_t>(kmax, ceil_div(d.K32, kOzChunkBlocks));
  }
  if (tiles == 0) return 1;
  const int64_t want = (2 * 152 + tiles - 1) / tiles;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, kmax));
}

// K split of each product: the requested one, but at least enough to keep
// every task within kOzMaxChunks exact chunks; a split product accumulates
// with atomics.  Returns whether any product accumulates (then its output
// must hold zeros or the value it accumulates onto before the launch).
bool set_ozaki_ksplit(std::vector<OzDesc>& descs, int ks, bool force_atomic) {
  bool any = false;
  for (OzDesc& g : descs) {
    g.ksplit = std::max(min_ozaki_ksplit(g), std::min(ks, std::max(1, ceil_div(g.K32, kOzChunkBlocks))));
    g.atomic = (force_atomic || g.ksplit > 1) ? 1 : 0;
    any = any || g.atomic;
  }
  return any;
}

void add_ozgemm_step(Plan& P, std::vector<OzDesc>& descs, int S, int level, bool force_atomic,
                     int ks, int slot, bool lower_c = false) {
  if (descs.empty()) return;
  std::vector<OzTask> tasks;
  double flops = 0, bytes = 0;
  set_ozaki_ksplit(descs, ks, force_atomic);
  for (size_t d = 0; d < descs.size(); d++) {
    OzDesc& g = descs[d];
    // the N tiles of one M block next to each other: they run in the same
    // wave and read the same A slices (the large operand, G), so A comes from
    // DRAM once and from L2 for the others
    for (int k = 0; k < g.ksplit; k++)
      for (int tm = 0; tm < ceil_div(g.M, 128); tm++)
        for (int tn = 0; tn < ceil_div(g.N, 64); tn++)
          if (!lower_c || (tm + 1) * 128 > tn * 64) tasks.push_back({(int)d, tm, tn, k});
    flops += (lower_c ? 1.0 : 2.0) * g.M * g.N * (double)g.K32 * 32;
    // slices of both operands read once, the FP64 result written (read too
    // when accumulated)
    bytes += 2.0 * S * ((double)g.M + g.N) * g.K32 * 32 +
             8.0 * g.M * g.N * (g.atomic ? 2.0 : 1.0) * g.cscale;
  }
  // longest tasks (most K blocks) first
  auto kblocks = [&](const OzTask& t) {
    const OzDesc& g = descs[t.d];
    int per = (g.K32 + g.ksplit - 1) / g.ksplit;
    per = (per + kOzChunkBlocks - 1) / kOzChunkBlocks * kOzChunkBlocks;
    return std::min(g.K32, (t.ks + 1) * per) - t.ks * per;
  };
  std::stable_sort(tasks.begin(), tasks.end(),
                   [&](const OzTask& a, const OzTask& b) { return kblocks(a) > kblocks(b); });
  Step st;
  st.kind = ST_OZGEMM;
  st.cfg = S;
  st.bytes = (size_t)bytes;
  st.n = (int)tasks.size();
  st.descs = P.push(descs);
  st.tasks = P.push(tasks);
  st.flops = flops;
  st.level = level;
  st.slot = slot;
  st.param = ks;
  gemm_features(st, descs, 32.0);
  P.steps.push_back(st);
}

// Scratch carving and descriptor helpers of the split-precision steps.
struct OzBuilder {
  pselinv_ctx* h;
  size_t off;  // next free byte of the scratch arena
  int S, cplx;
  OzBuilder(pselinv_ctx* h_, size_t off_)
      : h(h_), off(off_), S(h_->slices), cplx(h_->dtype == PSELINV_C128 ? 1 : 0) {}
  char* take(size_t bytes) {
    off = align256(off);
    const size_t o = off;
    off += bytes;
    h->scratch_high = std::max(h->scratch_high, off);
    return h->scratch + o;
  }
  // slice set of the R x Kd operand X: X(r, k) = src[r + k ld] (SLICE_ROWS)
  // or src[k + r ld] (SLICE_COLS)
  SliceDesc slice(const void* src, int ld, int mode, int R, int Kd) {
    SliceDesc d;
    d.src = (const double*)src;
    d.ld = ld;
    d.mode = mode;
    d.R = R;
    d.Kd = Kd;
    d.S = S;
    d.R64 = (int)r64(R);
    d.K32 = (int)k32(Kd) * (cplx ? 2 : 1);
    d.cplx = cplx;
    d.out = (__half*)take(slice_bytes(R, Kd, S) * (cplx ? 2 : 1));
    d.exps = (int*)take(exps_bytes(R));
    d.maxbits = nullptr;
    return d;
  }
  // one product (real) or two (real and imaginary parts) for C = alpha A B
  void product(std::vector<OzDesc>& out, const SliceDesc& a, const SliceDesc& b, char* C,
               int ldc, int M, int N, double alpha) const {
    OzDesc d{};
    d.alpha = alpha;
    d.A = a.out; d.eA = a.exps; d.A_R64 = a.R64;
    d.B = b.out; d.eB = b.exps; d.B_R64 = b.R64;
    d.C = (double*)C; d.ldc = ldc; d.M = M; d.N = N;
    d.K32 = a.K32;
    d.cscale = cplx ? 2 : 1;
    if (!cplx) {
      out.push_back(d);
      return;
    }
    d.half = a.K32 / 2;
    d.neg_half = 1;  // Re C = Re A Re B - Im A Im B
    d.coff = 0;
    out.push_back(d);
    d.neg_half = 0;  // Im C = Re A Im B + Im A Re B
    d.swap_b = 1;
    d.coff = 1;
    out.push_back(d);
  }
};

// Triangular solves of one factorisation level as sliced products (K = s):
// TL = AL Uinv (B(n, k) = Uinv(k, n)) and TU = AU Linv^T (B(n, k) =
// Linv(n, k)); Uinv and Linv hold exact zeros outside their triangles, so
// the full products are the triangular ones.  For symmetric values AU is AL
// and its slices serve both products.  Scratch from `base`.
void add_ozaki_trsm(pselinv_ctx* h, Plan& P, const std::vector<SchurProduct>& prods, int lev,
                    size_t base) {
  OzBuilder ob(h, base);
  int64_t nmax = 0;
  for (const SchurProduct& q : prods) nmax += q.c + q.cu + 2 * q.s;
  unsigned long long* maxbase = (unsigned long long*)ob.take((size_t)nmax * 8 + 8);
  std::vector<SliceDesc> sl;
  std::vector<OzDesc> out;
  int64_t moff = 0;
  for (const SchurProduct& q : prods) {
    SliceDesc al = ob.slice(q.AL, q.c, SLICE_ROWS, q.c, q.s);
    al.maxbits = maxbase + moff;
    SliceDesc ub = ob.slice(q.Uinv, q.s, SLICE_COLS, q.s, q.s);
    ub.maxbits = maxbase + moff + q.c;
    SliceDesc lb = ob.slice(q.Linv, q.s, SLICE_ROWS, q.s, q.s);
    lb.maxbits = maxbase + moff + q.c + q.s;
    SliceDesc au = al;
    if (q.AU != q.AL) {
      au = ob.slice(q.AU, q.cu, SLICE_ROWS, q.cu, q.s);
      au.maxbits = maxbase + moff + q.c + 2 * q.s;
      sl.push_back(au);
    }
    moff += q.c + q.cu + 2 * q.s;
    sl.push_back(al);
    sl.push_back(ub);
    sl.push_back(lb);
    ob.product(out, al, ub, q.TL, q.c, q.c, q.s, 1.0);
    ob.product(out, au, lb, q.TU, q.cu, q.cu, q.s, 1.0);
  }
  Step ms;
  ms.kind = ST_MEMSET;
  ms.ptr = maxbase;
  ms.bytes = (size_t)nmax * 8;
  ms.level = lev;
  P.steps.push_back(ms);
  add_slice_step(P, sl, lev, true);
  add_slice_step(P, sl, lev, false);
  add_ozgemm_step(P, out, h->slices, lev, false, 1, 0);
}

// Schur products of one factorisation level as sliced products: row maxima
// and slices of TL and TU (both by rows: A = TL, B = TU with K = s), then
// the products into the FP64 Sc blocks the scatter subtracts.  Scratch from
// `base` (bytes), after the level's FP64 region.
void add_ozaki_schur(pselinv_ctx* h, Plan& P, const std::vector<SchurProduct>& prods, int lev,
                     size_t base, bool lower) {
  OzBuilder ob(h, base);
  int64_t nmax = 0;
  for (const SchurProduct& q : prods) nmax += q.c + q.cu;
  unsigned long long* maxbase = (unsigned long long*)ob.take((size_t)nmax * 8 + 8);
  std::vector<SliceDesc> sl;
  std::vector<OzDesc> out;
  int64_t moff = 0;
  for (const SchurProduct& q : prods) {
    SliceDesc a = ob.slice(q.TL, q.c, SLICE_ROWS, q.c, q.s);
    a.maxbits = maxbase + moff;
    SliceDesc b = ob.slice(q.TU, q.cu, SLICE_ROWS, q.cu, q.s);
    b.maxbits = maxbase + moff + q.c;
    moff += q.c + q.cu;
    sl.push_back(a);
    sl.push_back(b);
    ob.product(out, a, b, q.Sc, q.c, q.c, q.cu, 1.0);
  }
  Step ms;
  ms.kind = ST_MEMSET;
  ms.ptr = maxbase;
  ms.bytes = (size_t)nmax * 8;
  ms.level = lev;
  P.steps.push_back(ms);
  add_slice_step(P, sl, lev, true);
  add_slice_step(P, sl, lev, false);
  // K = s <= 256 is one exact chunk: no K split, no accumulation
  add_ozgemm_step(P, out, h->slices, lev, false, 1, 0, lower);
}

// Split-precision normalisation of one depth level (Algorithm 1 step 2 and
// the diagonal block D_K = U_KK^{-1} L_KK^{-1} that starts Ainv_KK):
// Lhat = L_{C,K} Linv, Uhat^T = U_{K,C}^T Uinv^T and D_K = Uinv Linv as
// sliced products (K = s), after the maxima and slicing passes of the four
// operands (Linv and Uinv serve two products each).  Linv and Uinv hold
// exact zeros outside their triangles, so the full products are the
// triangular ones.  Steps go to the side stream; scratch from `base`.
void add_ozaki_normalize(pselinv_ctx* h, Plan& P, int lev, int64_t nb,
                         const std::vector<int64_t>& wbase, size_t base) {
  const HostSym& H = h->H;
  const size_t es = h->esize;
  OzBuilder ob(h, base);
  int64_t nmax = 0;
  for (int64_t b = 0; b < nb; b++)
    for (int64_t i = H.level_ptr[lev]; i < H.level_ptr[lev + 1]; i++) {
      const int64_t K = H.level_sn[i];
      nmax += 2 * cK(H, K) + 2 * H.sn_width[K];
    }
  if (nmax == 0) return;
  unsigned long long* maxbase = (unsigned long long*)ob.take(align256((size_t)nmax * 8 + 8));
  std::vector<SliceDesc> sl;
  std::vector<OzDesc> prods;
  int64_t moff = 0;
  for (int64_t b = 0; b < nb; b++)
    for (int64_t i = H.level_ptr[lev]; i < H.level_ptr[lev + 1]; i++) {
      const int64_t K = H.level_sn[i];
      const int s = (int)H.sn_width[K], c = (int)cK(H, K);
      const size_t so = ((size_t)b * H.storage + H.sn_offset[K]) * es;
      const size_t lo = so + (size_t)s * s * es, uo = lo + (size_t)c * s * es;
      const char* Linv = h->scratch + (size_t)wbase[b * H.ns + K] * es;
      const char* Uinv = Linv + (size_t)s * s * es;
      SliceDesc lb = ob.slice(Linv, s, SLICE_COLS, s, s);  // Linv(k, n)
      SliceDesc ub = ob.slice(Uinv, s, SLICE_ROWS, s, s);  // Uinv(n, k) = Uinv(m, k)
      lb.maxbits = maxbase + moff;
      ub.maxbits = maxbase + moff + s;
      moff += 2 * s;
      sl.push_back(lb);
      sl.push_back(ub);
      ob.product(prods, ub, lb, h->ainv + so, s, s, s, 1.0);  // D_K
      if (c == 0) continue;
      SliceDesc la = ob.slice(h->lu + lo, c, SLICE_ROWS, c, s);  // L_{C,K}(m, k)
      la.maxbits = maxbase + moff;
      sl.push_back(la);
      ob.product(prods, la, lb, h->nf + lo, c, c, s, 1.0);
      if (!h->opts.symmetric) {  // symmetric A: Uhat = Lhat^T, not needed
        SliceDesc ua = ob.slice(h->lu + uo, c, SLICE_ROWS, c, s);  // U_{K,C}^T(m, k)
        ua.maxbits = maxbase + moff + c;
        sl.push_back(ua);
        ob.product(prods, ua, ub, h->nf + uo, c, c, s, 1.0);
      }
      moff += 2 * c;
    }
  const size_t first = P.steps.size();
  Step ms;
  ms.kind = ST_MEMSET;
  ms.ptr = maxbase;
  ms.bytes = (size_t)nmax * 8;
  ms.level = lev;
  P.steps.push_back(ms);
  add_slice_step(P, sl, lev, true);
  add_slice_step(P, sl, lev, false);
  add_ozgemm_step(P, prods, h->slices, lev, false, 1, -1);
  for (size_t i = first; i < P.steps.size(); i++) P.steps[i].side = 1;
}

// Merge the finished blocks of the supernodes `sns` (diagonal block, L and
// U^T panels of every instance) into the running row / column maxima of
// Ainv: what a later level's G reads is bounded by them.
void add_outmax_step(pselinv_ctx* h, Plan& P, const std::vector<int64_t>& sns, int lev) {
  const HostSym& H = h->H;
  std::vector<MaxTask> tasks;
  for (int64_t b = 0; b < h->nbatch; b++)
    for (int64_t K : sns) {
      const int s = (int)H.sn_width[K], c = (int)cK(H, K), cu = (int)cU(H, K);
      const int64_t so = H.sn_offset[K];
      // L panel: rows of Ainv (R_K) for a structurally symmetric handle,
      // columns (R_L) for a general one; the U^T panel the other way round
      const int lwhich = H.general ? 2 : 1, uwhich = H.general ? 1 : 2;
      for (int r = 0; r < ceil_div(s, kOutMaxRows); r++) tasks.push_back({(int)b, (int)K, 0, r, so, s, 0});
      for (int r = 0; r < ceil_div(c, kOutMaxRows); r++)
        tasks.push_back({(int)b, (int)K, lwhich, r, so + (int64_t)s * s, c, 0});
      for (int r = 0; r < ceil_div(cu, kOutMaxRows); r++)
        tasks.push_back({(int)b, (int)K, uwhich, r, so + (int64_t)s * s + (int64_t)c * s, cu,
                         H.general ? 1 : 0});
    }
  if (tasks.empty()) return;
  Step st;
  st.kind = ST_OUTMAX;
  st.n = (int)tasks.size();
  st.tasks = P.push(tasks);
  double bytes = 0;
  for (int64_t K : sns) {
    const double s = (double)H.sn_width[K];
    bytes += s * (s + cK(H, K) + cU(H, K));
  }
  st.bytes = (size_t)(bytes * h->nbatch * h->esize);
  st.level = lev;
  P.steps.push_back(st);
}

// One level (or one supernode) of the split-precision sweep: gather G,
// slice G (by rows and by columns), Lhat and Uhat^T, sliced products for
// steps 3 and 5, slice Ainv(C,K), sliced product for step 4 accumulated onto
// D_K.  Scratch layout after the W region (byte offsets).
void add_ozaki_level(pselinv_ctx* h, Plan& P, const std::vector<int64_t>& grp, int64_t nb,
                     int64_t gbase_scalars, int lev, size_t& max_cursor) {
  const HostSym& H = h->H;
  const int S = h->slices;
  const size_t es = h->esize;
  const int cplx = h->dtype == PSELINV_C128 ? 1 : 0;
  std::vector<SliceDesc> gd, sl2;  // gd: G by rows / columns, Lhat, Uhat^T of every supernode
  std::vector<GTileTask> gt;
  std::vector<int> dense;          // the panels' slice sets in gd
  std::vector<OzDesc> main, dg;
  std::vector<CopySeg> zero, mirror;
  const bool sym = h->opts.symmetric != 0;
  OzBuilder ob(h, (size_t)gbase_scalars * es);
  // column maxima of every panel operand of the level (the sweep's maxima
  // region, zeroed at its start); G's exponents come from the running
  // row / column maxima of Ainv instead
  int64_t nmax = 0;
  for (int64_t b = 0; b < nb; b++)
    for (int64_t K : grp)
      if (cK(H, K) > 0 && cU(H, K) > 0) nmax += 3 * H.sn_width[K];
  std::vector<CopySeg> zside;  // general patterns: a panel whose products are empty
  for (int64_t b = 0; b < nb; b++)
    for (int64_t K : grp)
      if ((cK(H, K) == 0) != (cU(H, K) == 0)) {
        const size_t so = ((size_t)b * H.storage + H.sn_offset[K]) * es;
        zside.push_back({nullptr, h->ainv + so + (size_t)H.sn_width[K] * H.sn_width[K] * es,
                         (cK(H, K) + cU(H, K)) * H.sn_width[K] * (cplx ? 2 : 1)});
      }
  add_zero_step(P, zside, lev);
  if (nmax == 0) return;  // roots only (c = 0): nothing after D_K
  unsigned long long* maxbase = (unsigned long long*)(h->scratch + max_cursor);
  max_cursor += align256((size_t)nmax * 8 + 8);
  h->scratch_high = std::max(h->scratch_high, max_cursor);
  int64_t moff = 0;
  auto push_product = [&](std::vector<OzDesc>& out, const SliceDesc& a, const SliceDesc& b,
                          char* C, int ldc, int M, int N) {
    ob.product(out, a, b, C, ldc, M, N, -1.0);
  };
  for (int64_t b = 0; b < nb; b++)
    for (int64_t K : grp) {
      // c: rows of the L panel (R_L(K) = R_K), cu: rows of the U^T panel
      // (R_U(K) for a general pattern, else c); G = Ainv(R_U, R_L) is cu x c
      const int s = (int)H.sn_width[K], c = (int)cK(H, K), cu = (int)cU(H, K);
      if (c == 0 || cu == 0) continue;
      const int64_t m0 = moff;
      moff += 3 * s;
      const size_t so = ((size_t)b * H.storage + H.sn_offset[K]) * es;
      const size_t lo = so + (size_t)s * s * es, uo = lo + (size_t)c * s * es;
      // symmetric A: G is symmetric and Uhat = Lhat^T, so step 5's product is
      // the transpose of step 3's (a copy) and step 4 uses Lhat
      SliceDesc gr = ob.slice(nullptr, cu, SLICE_ROWS, cu, c);  // G by rows (from the gather)
      SliceDesc lh = ob.slice(h->nf + lo, c, SLICE_COLS, s, c);
      lh.maxbits = maxbase + m0;
      SliceDesc gc = gr, uh = lh;
      if (!sym) {
        gc = ob.slice(nullptr, c, SLICE_COLS, c, cu);  // G by columns
        uh = ob.slice(h->nf + uo, cu, SLICE_COLS, s, cu);
        uh.maxbits = maxbase + m0 + s;
      }
      // Ainv(R_U, K): the U^T panel of a general pattern, the L panel otherwise
      char* ainv_uk = H.general ? h->ainv + uo : h->ainv + lo;
      char* ainv_kl = H.general ? h->ainv + lo : h->ainv + uo;
      SliceDesc ak = ob.slice(ainv_uk, cu, SLICE_COLS, s, cu);
      ak.maxbits = maxbase + m0 + 2 * s;
      const int ir = (int)gd.size();
      gd.push_back(gr);
      const int ic = sym ? -1 : (int)gd.size();
      if (!sym) gd.push_back(gc);
      dense.push_back((int)gd.size());
      gd.push_back(lh);
      if (!sym) {
        dense.push_back((int)gd.size());
        gd.push_back(uh);
      }
      for (int tq = 0; tq < ceil_div(c, 64); tq++)
        for (int tp = 0; tp < ceil_div(cu, 64); tp++)
          gt.push_back({(int)b, (int)K, tp, tq, ir, ic});
      sl2.push_back(ak);
      // step 3: Ainv(R_U, K) = -G Lhat;  step 5: Ainv(K, R_L)^T = -G^T Uhat^T
      push_product(main, gr, lh, ainv_uk, cu, cu, s);
      if (!sym) push_product(main, gc, uh, ainv_kl, c, c, s);
      else mirror.push_back({h->ainv + lo, h->ainv + uo, (int64_t)c * s});
      // step 4: Ainv(K,K) = D_K - Uhat Ainv(R_U, K)
      push_product(dg, uh, ak, h->ainv + so, s, s, s);
      zero.push_back({nullptr, h->ainv + lo, (int64_t)(c + cu) * s * (cplx ? 2 : 1)});
    }
  if (gt.empty()) return;
  const int prec = PSELINV_PREC_OZAKI_FP16;
  const int ks_main = tuned_value(h, prec, lev, 1, choose_ozaki_ksplit(main));
  const int ks_diag = tuned_value(h, prec, lev, 2, choose_ozaki_ksplit(dg));
  // the panels' maxima, then G's slices in both layouts straight from the
  // ancestors' blocks (exponents from the running maxima of Ainv) with the
  // panels' slices in the same launch
  add_gslice_step(P, gd, {}, dense, lev, true, es);
  add_gslice_step(P, gd, gt, dense, lev, false, es);
  // outputs of products split along K (requested, or forced by the exact
  // chunk limit) are accumulated: zero them first
  if (set_ozaki_ksplit(main, ks_main, false)) add_zero_step(P, zero, lev);
  add_ozgemm_step(P, main, S, lev, false, ks_main, 1);
  add_copy_step(P, mirror, lev, es);
  add_slice_step(P, sl2, lev, true);
  add_slice_step(P, sl2, lev, false);
  add_ozgemm_step(P, dg, S, lev, true, ks_diag, 2);
}

// largest K split of the normalisation's products
constexpr int kNormMaxKsplit = 8;
// triangular-inverse tasks (8 columns each) of the levels whose inverses
// the side stream computes itself, and of the first third-stream launch
constexpr int64_t kTriSideTasks = 4 * 152;
constexpr int64_t kTriThirdTasks = 8 * 152;

// An FP64 level of narrow supernodes as one fused launch (gather and steps
// 3-5 in shared memory), each supernode's output columns split into tasks
// of at most kSmallLevelTaskFma multiply-adds, when every supernode fits
// and the estimated time (multiply-adds at 2 per cycle and SM) is below
// that of the gather and two GEMM launches (about 15 us each plus the
// level's flops at 1 TFLOP/s).  Returns false to leave
// the level to those launches.
constexpr double kSmallLevelTaskFma = 65536;
bool add_small_level(pselinv_ctx* h, Plan& P, const std::vector<int64_t>& grp, int64_t nb, int lev) {
  const HostSym& H = h->H;
  const bool sym = h->opts.symmetric != 0;
  const double cplx = h->dtype == DT_F64 ? 1.0 : 4.0;
  std::vector<SnTask> tasks;
  size_t smem = 0;
  double fma_max = 0, flops = 0, bytes = 0;
  for (int64_t K : grp) {
    const int64_t s = H.sn_width[K], c = cK(H, K);
    if (c == 0) continue;
    if (c > kSmallLevelMaxC) return false;
    // multiply-adds per output column: steps 3 and 5 (c^2 each), step 4 (s c)
    const double per_col = cplx * ((sym ? 1.0 : 2.0) * c * c + (double)s * c);
    const int w = (int)std::max<int64_t>(1, std::min<int64_t>(s, (int64_t)(kSmallLevelTaskFma / per_col)));
    const int64_t rb = H.rows_ptr[K], b0 = H.rows_blk[rb], bl = H.rows_blk[rb + c - 1];
    const int64_t seg = H.blk_rel[bl] + (c - H.blk_pb[bl]) - H.blk_rel[b0];
    const size_t b = small_level_smem(h->dtype, (int)c, (int)s, w, (int)(bl - b0 + 1), (int)seg);
    if (b > kSmallLevelMaxSmem) return false;
    smem = std::max(smem, b);
    fma_max = std::max(fma_max, per_col * w);
    flops += 2.0 * per_col * s * nb;
    bytes += (double)h->esize * nb * (c * c + 4.0 * c * s + 2.0 * s * s);
    for (int64_t b2 = 0; b2 < nb; b2++)
      for (int64_t j0 = 0; j0 < s; j0 += w)
        tasks.push_back({(int)b2, (int)K, (int)j0, (int)std::min<int64_t>(w, s - j0)});
  }
  if (tasks.empty()) return false;
  // the largest task alone on an SM, or the level's multiply-adds spread
  // over all 152 SMs, whichever is longer
  const double t_fused = std::max(fma_max, flops / 2.0 / 152.0) / 2.0 / 2.07e9;
  const double t_launches = 3 * 15e-6 + flops / 1e12;
  if (t_fused >= t_launches) return false;
  Step st;
  st.kind = ST_SMALL_LEVEL;
  st.cfg = (int)smem;
  st.n = (int)tasks.size();
  st.tasks = P.push(tasks);
  st.flops = flops;
  st.bytes = (size_t)bytes;
  st.level = lev;
  P.steps.push_back(st);
  return true;
}

// FP64-equivalent flops of the products of steps 3-5 of depth level `lev`
// over every instance (sum 4 c^2 s; x4 for complex)
double level_product_flops(const pselinv_ctx* h, int lev) {
  const HostSym& H = h->H;
  double lf = 0;
  for (int64_t i = H.level_ptr[lev]; i < H.level_ptr[lev + 1]; i++) {
    const double c = (double)cK(H, H.level_sn[i]), w = (double)H.sn_width[H.level_sn[i]];
    lf += 4.0 * c * (double)cU(H, H.level_sn[i]) * w;
  }
  return lf * (double)h->nbatch * (h->dtype == DT_F64 ? 1.0 : 4.0);
}

int build_selinv_plan(pselinv_ctx* h, int schedule, int precision) {
  const HostSym& H = h->H;
  const bool sym = h->opts.symmetric != 0;
  Plan& P = h->selinv_plan[precision][schedule];
  P.release();
  h->scratch_high = 0;
  const size_t es = h->esize;
  const int dt = h->dtype;
  const int64_t nb = h->nbatch;
  const int cfg = choose_cfg(schedule);
  // W region: Linv | Uinv per (instance, supernode)
  std::vector<int64_t> wbase((size_t)(nb * H.ns));
  int64_t off = 0;
  for (int64_t b = 0; b < nb; b++)
    for (int64_t K = 0; K < H.ns; K++) {
      wbase[b * H.ns + K] = off;
      off += 2 * H.sn_width[K] * H.sn_width[K];
    }
  const int64_t gbase = off;
  // Normalisation (Algorithm 1 step 2 and D_K) on the side stream, one
  // depth level ahead of the sweep so that it overlaps the previous level's
  // products.  Triangular inverses first: the blocks of the levels nearest
  // the roots (needed first, few and wide) in one launch on the side
  // stream; the next levels' in a launch on a third stream that runs beside
  // the first levels, and the deep levels' in a second one behind it; the
  // first normalisation that needs either waits for it.
  const int nlev = (int)H.level_ptr.size() - 1;
  // a partitioned sweep covers a subset of the supernodes
  auto in_set = [&](int64_t K) { return h->subset.empty() || h->subset[(size_t)K] != 0; };
  int lev_a = -1, lev_b = -1;
  {
    auto level_tasks = [&](int l) {
      int64_t t = 0;
      for (int64_t i = H.level_ptr[l]; i < H.level_ptr[l + 1]; i++)
        t += 2 * ((H.sn_width[H.level_sn[i]] + 7) / 8);
      return t * nb;
    };
    int64_t tasks = 0;
    for (int l = 0; l < nlev; l++) {
      if (l > 0 && tasks + level_tasks(l) > kTriSideTasks) break;
      tasks += level_tasks(l);
      lev_a = l;
    }
    tasks = 0;
    lev_b = lev_a;
    for (int l = lev_a + 1; l < nlev; l++) {
      if (l > lev_a + 1 && tasks + level_tasks(l) > kTriThirdTasks) break;
      tasks += level_tasks(l);
      lev_b = l;
    }
    std::vector<TriBlock> ta, tb, tc;
    for (int64_t b = 0; b < nb; b++)
      for (int l = 0; l < nlev; l++)
        for (int64_t i = H.level_ptr[l]; i < H.level_ptr[l + 1]; i++) {
          const int64_t K = H.level_sn[i];
          if (!in_set(K)) continue;
          (l <= lev_a ? ta : l <= lev_b ? tb : tc).push_back({b, K, wbase[b * H.ns + K]});
        }
    add_tri_step(P, H, ta, -1, 1, false);  // one launch: the first normalisation waits for it
    add_tri_step(P, H, tb, -1, 2);
    if (!tb.empty()) P.steps.back().signal = EV_THIRD_DONE;
    add_tri_step(P, H, tc, -1, 2);
    if (!tc.empty()) P.steps.back().signal = EV_THIRD_DONE2;
  }
  const size_t norm_base = selinv_main_bytes(H, nb, es);
  const size_t max_base = norm_base + ozaki_norm_bytes(H, nb, 6, es);
  size_t max_cursor = max_base;
  bool third_waited = false, third_waited2 = false;
  // split = true: Lhat, Uhat^T and D_K as sliced products
  auto add_normalize = [&](int lev, bool split) {
    std::vector<GemmDesc> norm;
    for (int64_t b = 0; b < nb; b++)
      for (int64_t i = H.level_ptr[lev]; i < H.level_ptr[lev + 1]; i++) {
        const int64_t K = H.level_sn[i];
        if (!in_set(K)) continue;
        const int64_t s = H.sn_width[K], c = cK(H, K), cu = cU(H, K), w0 = wbase[b * H.ns + K];
        const size_t so = ((size_t)b * H.storage + H.sn_offset[K]) * es;
        char* Linv = h->scratch + (size_t)w0 * es;
        char* Uinv = Linv + (size_t)s * s * es;
        if (split) continue;  // all three as sliced products
        // D_K = Uinv Linv (upper x lower), Lhat = L Linv, Uhat^T = U^T Uinv^T (lower B)
        norm.push_back(make_desc(Uinv, Linv, h->ainv + so, s, s, s, s, s, s, 0, 0, 1.0, 0.0, 0, 1,
                                 GEMM_TRI_UPPER_A | GEMM_TRI_LOWER_B));
        const size_t lo = so + (size_t)s * s * es, uo = lo + (size_t)c * s * es;
        if (c > 0)
          norm.push_back(make_desc(h->lu + lo, Linv, h->nf + lo, c, s, s, c, s, c, 0, 0, 1.0, 0.0,
                                   0, 1, GEMM_TRI_LOWER_B));
        if (cu > 0 && !h->opts.symmetric)  // symmetric A: Uhat = Lhat^T, not needed
          norm.push_back(make_desc(h->lu + uo, Uinv, h->nf + uo, cu, s, s, cu, s, cu, 0, 1, 1.0,
                                   0.0, 0, 1, GEMM_TRI_LOWER_B));
      }
    const size_t first = P.steps.size();
    // levels of few wide supernodes (near the roots): split K so that the
    // launch has tasks for every SM, its K loops being the level's latency;
    // the outputs are then zeroed and accumulated
    int64_t ntask = 0, kmax = 0;
    for (const GemmDesc& g : norm) {
      ntask += (int64_t)ceil_div(g.M, kRowsBlock) * ceil_div(g.N, kRowsChunk);
      kmax = std::max<int64_t>(kmax, g.K);
    }
    int ks = 1;
    while (ks < kNormMaxKsplit && ntask * ks < 152 * 8 && kmax / (2 * ks) >= 32) ks *= 2;
    if (ks > 1) {
      std::vector<CopySeg> zero;
      for (GemmDesc& g : norm) {
        g.ksplit = ks;
        g.atomic = 1;
        zero.push_back({nullptr, g.C, (int64_t)g.M * g.N * (int64_t)(es / 8)});
      }
      add_zero_step(P, zero, lev);
    }
    add_gemm_step(P, dt, tuned_value(h, precision, lev, 0, GEMM_ROWS), norm, lev, 0);
    if (split) add_ozaki_normalize(h, P, lev, nb, wbase, norm_base);
    for (size_t i = first; i < P.steps.size(); i++) P.steps[i].side = 1;
    if (P.steps.size() > first) {
      if (lev > lev_b && !third_waited2) {
        P.steps[first].wait = EV_THIRD_DONE2;  // after EV_THIRD_DONE on the same stream
        third_waited = third_waited2 = true;
      } else if (lev > lev_a && !third_waited) {
        P.steps[first].wait = EV_THIRD_DONE;
        third_waited = true;
      }
      P.steps.back().signal = EV_LEVEL + lev;
    }
  };
  P.two_streams = true;
  P.ev.assign(EV_LEVEL + std::max(nlev, 0), nullptr);
  for (auto& e : P.ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  // split precision: each level runs either the sliced tensor-core products
  // (normalisation included) or, for levels whose products are too small
  // to pay for the slicing, the FP64 ones; the default is a flop
  // threshold, the tuner times both
  std::vector<char> split_lv((size_t)std::max(nlev, 0), 0);
  int last_split = -1;  // the running maxima are kept up to this level
  for (int lev = 0; lev < nlev; lev++) {
    if (precision != PSELINV_PREC_OZAKI_FP16) break;
    const int mode = tuned_value(h, precision, lev, 3, level_product_flops(h, lev) < 2e8 ? 1 : 0);
    split_lv[(size_t)lev] = mode == 0;
    if (mode == 0) last_split = lev;
  }
  for (size_t lev = 0; lev + 1 < H.level_ptr.size(); lev++) {
    const bool split_level = split_lv[lev] != 0;
    add_normalize((int)lev, split_level && h->opts.split_normalise != 0 && !H.general);
    const size_t first_main = P.steps.size();
    // groups: the whole level, or one supernode at a time
    std::vector<std::vector<int64_t>> groups;
    if (schedule == PSELINV_SCHED_LEVEL) {
      groups.emplace_back();
      for (int64_t i = H.level_ptr[lev]; i < H.level_ptr[lev + 1]; i++)
        if (in_set(H.level_sn[i])) groups.back().push_back(H.level_sn[i]);
      if (groups.back().empty()) groups.pop_back();
    } else {
      for (int64_t i = H.level_ptr[lev]; i < H.level_ptr[lev + 1]; i++)
        if (in_set(H.level_sn[i])) groups.push_back({H.level_sn[i]});
    }
    const int slot_main = precision == PSELINV_PREC_OZAKI_FP16 ? 4 : 1;
    const int slot_diag = precision == PSELINV_PREC_OZAKI_FP16 ? 5 : 2;
    for (const auto& grp : groups) {
      if (split_level) {
        add_ozaki_level(h, P, grp, nb, gbase, (int)lev, max_cursor);
        continue;
      }
      if (schedule == PSELINV_SCHED_LEVEL && !H.general && add_small_level(h, P, grp, nb, (int)lev))
        continue;
      std::vector<SnTask> gt;
      std::vector<int64_t> gofs;
      std::vector<GemmDesc> main, dg;
      std::vector<CopySeg> mirror, zsegs;
      int64_t goff = gbase;
      for (int64_t b = 0; b < nb; b++)
        for (int64_t K : grp) {
          const int64_t s = H.sn_width[K], c = cK(H, K), cu = cU(H, K);
          if (c == 0 || cu == 0) {
            // nothing after D_K; with one structure empty (a general
            // pattern) the other panel of Ainv is zero (steps 3 and 5 sum
            // over the empty one)
            if (c + cu > 0) {
              const size_t so = ((size_t)b * H.storage + H.sn_offset[K]) * es;
              zsegs.push_back({nullptr, h->ainv + so + (size_t)s * s * es,
                               (c + cu) * s * (int64_t)(es / 8)});
            }
            continue;
          }
          const int64_t g0 = goff;
          goff += c * cu;
          h->scratch_high = std::max(h->scratch_high, (size_t)goff * es);
          const size_t so = ((size_t)b * H.storage + H.sn_offset[K]) * es;
          const size_t lo = so + (size_t)s * s * es, uo = lo + (size_t)c * s * es;
          char* G = h->scratch + (size_t)g0 * es;
          const int ksplit = std::max(1, (int)std::min<int64_t>(cu / 256, 64));
          if (H.general) {
            // G = Ainv(R_U, R_L) (cu x c).  Step 3: Ainv(R_U, K) = -G Lhat into
            // the U^T panel; step 5: Ainv(K, R_L)^T = -G^T Uhat^T into the L
            // panel; step 4: Ainv_KK += -Uhat Ainv(R_U, K)
            for (int tq = 0; tq < ceil_div(c, 32); tq++)
              for (int tp = 0; tp < ceil_div(cu, 32); tp++) {
                gt.push_back({(int)b, (int)K, tp, tq});
                gofs.push_back(g0);
              }
            main.push_back(make_desc(G, h->nf + lo, h->ainv + uo, cu, s, c, cu, c, cu, 0, 0, -1.0, 0.0));
            main.push_back(make_desc(G, h->nf + uo, h->ainv + lo, c, s, cu, cu, cu, c, 1, 0, -1.0, 0.0));
            dg.push_back(make_desc(h->nf + uo, h->ainv + uo, h->ainv + so, s, s, cu, cu, cu, s, 1, 0,
                                   -1.0, 1.0, 1, ksplit));
            continue;
          }
          for (int tq = 0; tq < ceil_div(c, 32); tq++)
            for (int tp = 0; tp < ceil_div(c, 32); tp++) {
              gt.push_back({(int)b, (int)K, tp, tq});
              gofs.push_back(g0);
            }
          main.push_back(make_desc(G, h->nf + lo, h->ainv + lo, c, s, c, c, c, c, 0, 0, -1.0, 0.0));
          // symmetric A: step 5 is the transpose of step 3 and Uhat = Lhat^T
          if (sym)
            mirror.push_back({h->ainv + lo, h->ainv + uo, c * s});
          else
            main.push_back(make_desc(G, h->nf + uo, h->ainv + uo, c, s, c, c, c, c, 1, 0, -1.0, 0.0));
          dg.push_back(make_desc(h->nf + (sym ? lo : uo), h->ainv + lo, h->ainv + so, s, s, c, c, c,
                                 s, 1, 0, -1.0, 1.0, 1, ksplit));
        }
      add_zero_step(P, zsegs, (int)lev);
      if (gt.empty()) continue;
      Step g;
      g.kind = ST_GATHER;
      g.bytes = (size_t)((goff - gbase) * (int64_t)es * 2);
      g.n = (int)gt.size();
      g.tasks = P.push(gt);
      g.offs = P.push(gofs);
      g.level = (int)lev;
      P.steps.push_back(g);
      add_gemm_step(P, dt, tuned_value(h, precision, (int)lev, slot_main, cfg), main, (int)lev,
                    slot_main);
      add_copy_step(P, mirror, (int)lev, es);
      add_gemm_step(P, dt, tuned_value(h, precision, (int)lev, slot_diag, cfg), dg, (int)lev,
                    slot_diag);
    }
    if ((int)lev < last_split) {  // a later split level slices blocks of this one
      std::vector<int64_t> sns;
      for (int64_t i = H.level_ptr[lev]; i < H.level_ptr[lev + 1]; i++)
        if (in_set(H.level_sn[i])) sns.push_back(H.level_sn[i]);
      add_outmax_step(h, P, sns, (int)lev);
    }
    if (P.steps.size() > first_main) P.steps[first_main].wait = EV_LEVEL + (int)lev;
  }
  if (last_split >= 0) {
    // a partitioned sweep starts from imported blocks G_r = Ainv(R_U(r),
    // R_L(r)) of its subtree roots r: their row and column maxima first
    std::vector<GTileTask> roots;
    for (int64_t b = 0; b < nb; b++)
      for (int64_t K = 0; K < H.ns && !h->subset.empty(); K++) {
        const int64_t par = H.sn_parent[K];
        if (!in_set(K) || par < 0 || in_set(par) || cK(H, K) == 0 || cU(H, K) == 0) continue;
        for (int tq = 0; tq < ceil_div(cK(H, K), 64); tq++)
          for (int tp = 0; tp < ceil_div(cU(H, K), 64); tp++)
            roots.push_back({(int)b, (int)K, tp, tq, 0, -1});
      }
    std::vector<Step> pre;
    Step ms;
    ms.kind = ST_MEMSET;
    ms.ptr = h->rcmax;
    ms.bytes = (size_t)nb * 2 * H.n * 8;
    pre.push_back(ms);
    if (!roots.empty()) {
      std::vector<SliceDesc> none(1);
      const size_t at = P.steps.size();
      add_gslice_step(P, none, roots, {}, -1, true, es);
      pre.push_back(P.steps[at]);
      P.steps.pop_back();
    }
    P.steps.insert(P.steps.begin(), pre.begin(), pre.end());
  }
  // the scratch sizes above bound every region the steps use
  if (h->scratch_high > h->scratch_bytes) return PSELINV_ERR_CHECK;
  if (max_cursor > max_base) {  // one memset of every split level's maxima, first on the sweep
    Step ms;
    ms.kind = ST_MEMSET;
    ms.ptr = h->scratch + max_base;
    ms.bytes = max_cursor - max_base;
    P.steps.insert(P.steps.begin(), ms);
  }
  CK(cudaMalloc(&P.arena, P.host.size() + 256));
  CK(cudaMemcpy(P.arena, P.host.data(), P.host.size(), cudaMemcpyHostToDevice));
  P.built = true;
  return PSELINV_OK;
}

void launch_step(pselinv_ctx* h, const Plan& P, const Step& s, cudaStream_t st) {
  char* a = P.arena;
  switch (s.kind) {
    case ST_GEMM:
      launch_gemm(h->dtype, s.cfg, (const GemmDesc*)(a + s.descs), (const GemmTask*)(a + s.tasks),
                  s.n, s.grid, st);
      break;
    case ST_TRI_INV:
      launch_tri_inv(h->dtype, h->S, h->lu, h->scratch, (const int64_t*)(a + s.offs),
                     (const SnTask*)(a + s.tasks), s.n, h->max_width, s.cfg, st);
      break;
    case ST_LU_PANEL:
      launch_lu_panel(h->dtype, h->S, h->lu, (const SnTask*)(a + s.tasks), s.n, st);
      break;
    case ST_GATHER:
      if (h->H.general)
        launch_gather_general(h->dtype, h->S, h->ainv, h->scratch, (const int64_t*)(a + s.offs),
                              (const SnTask*)(a + s.tasks), s.n, st);
      else
        launch_gather(h->dtype, h->S, h->ainv, h->scratch, (const int64_t*)(a + s.offs),
                      (const SnTask*)(a + s.tasks), s.n, st,
                      s.ptr2 ? (const int64_t*)(a + s.offs2) : nullptr,
                      (unsigned long long*)s.ptr2);
      break;
    case ST_SCATTER_SUB:
      if (h->H.general)
        launch_scatter_sub_general(h->dtype, h->S, h->lu, h->scratch, (const int64_t*)(a + s.offs),
                                   (const SnTask*)(a + s.tasks), s.n, st);
      else
        launch_scatter_sub(h->dtype, h->S, h->lu, h->scratch, (const int64_t*)(a + s.offs),
                           (const SnTask*)(a + s.tasks), s.n, s.cfg == 1, st);
      break;
    case ST_COPY:
      launch_copy(h->dtype, (const CopySeg*)(a + s.tasks), s.n, s.grid, st);
      break;
    case ST_MEMSET:
      cudaMemsetAsync(s.ptr, 0, s.bytes, st);
      break;
    case ST_SCATTER_VALUES:
      launch_scatter_values(h->dtype, h->S, h->staging, h->lu, (int)h->nbatch, st);
      break;
    case ST_SLICE:
      launch_slice((const SliceDesc*)(a + s.descs), (const SliceTask*)(a + s.tasks), s.n,
                   s.cfg == 1, st);
      break;
    case ST_OZGEMM:
      launch_ozaki_gemm(s.cfg, (const OzDesc*)(a + s.descs), (const OzTask*)(a + s.tasks), s.n,
                        h->derr, s.side == 0, h->opts.ozaki_a_tmem != 0, st);
      break;
    case ST_ZERO:
      launch_zero((const CopySeg*)(a + s.tasks), s.n, s.grid, st);
      break;
    case ST_SMALL_LEVEL:
      launch_small_level(h->dtype, h->S, h->ainv, h->nf, (const SnTask*)(a + s.tasks), s.n,
                         (size_t)s.cfg, h->opts.symmetric != 0, st);
      break;
    case ST_GSLICE:
      launch_gslice(h->dtype, h->S, h->ainv, (const SliceDesc*)(a + s.descs),
                    (const GTileTask*)(a + s.tasks), s.n, (const SliceTask*)(a + s.offs), s.n2,
                    s.cfg == 1, h->rcmax, st);
      break;
    case ST_MIRROR:
      launch_mirror_lower(h->dtype, h->S, h->lu, (const SnTask*)(a + s.tasks), s.n, st);
      break;
    case ST_OUTMAX:
      launch_out_maxima(h->dtype, h->S, h->ainv, (const MaxTask*)(a + s.tasks), s.n, h->rcmax, st);
      break;
  }
}

// The streams of a multi-stream sweep (created on first use): the sweep's
// own launches at the highest priority, the normalisation one level ahead
// below it, the triangular inverses of the deeper levels lowest, so that
// pending CTAs of the critical path are scheduled first.
struct SweepStreams {
  cudaStream_t main, side, third;
};
int sweep_streams(pselinv_ctx* h, SweepStreams* out) {
  int least = 0, greatest = 0;
  CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  const int middle = least + (greatest - least) / 2;
  if (!h->main_stream)
    CK(cudaStreamCreateWithPriority(&h->main_stream, cudaStreamNonBlocking, greatest));
  if (!h->side_stream)
    CK(cudaStreamCreateWithPriority(&h->side_stream, cudaStreamNonBlocking, middle));
  if (!h->third_stream)
    CK(cudaStreamCreateWithPriority(&h->third_stream, cudaStreamNonBlocking, least));
  *out = {h->main_stream, h->side_stream, h->third_stream};
  return PSELINV_OK;
}

// Issue the plan on `st`; steps marked `side` go to the side stream, forked
// from and joined back into `st` with events (also inside a graph capture).
int run_steps(pselinv_ctx* h, Plan& P, cudaStream_t st) {
  if (!P.two_streams) {
    for (const Step& s : P.steps) launch_step(h, P, s, st);
    CK(cudaGetLastError());
    return PSELINV_OK;
  }
  SweepStreams q3;
  const int rc = sweep_streams(h, &q3);
  if (rc != PSELINV_OK) return rc;
  CK(cudaEventRecord(P.ev[EV_FORK], st));
  CK(cudaStreamWaitEvent(q3.main, P.ev[EV_FORK], 0));
  CK(cudaStreamWaitEvent(q3.side, P.ev[EV_FORK], 0));
  CK(cudaStreamWaitEvent(q3.third, P.ev[EV_FORK], 0));
  for (const Step& s : P.steps) {
    cudaStream_t q = s.side == 1 ? q3.side : s.side == 2 ? q3.third : q3.main;
    if (s.wait >= 0) CK(cudaStreamWaitEvent(q, P.ev[s.wait], 0));
    launch_step(h, P, s, q);
    if (s.signal >= 0) CK(cudaEventRecord(P.ev[s.signal], q));
  }
  CK(cudaEventRecord(P.ev[EV_MAIN_JOIN], q3.main));
  CK(cudaEventRecord(P.ev[EV_SIDE_JOIN], q3.side));
  CK(cudaEventRecord(P.ev[EV_THIRD_JOIN], q3.third));
  CK(cudaStreamWaitEvent(st, P.ev[EV_MAIN_JOIN], 0));
  CK(cudaStreamWaitEvent(st, P.ev[EV_SIDE_JOIN], 0));
  CK(cudaStreamWaitEvent(st, P.ev[EV_THIRD_JOIN], 0));
  CK(cudaGetLastError());
  return PSELINV_OK;
}

int run_plan(pselinv_ctx* h, Plan& P, cudaStream_t st, bool graph) {
  if (!graph) return run_steps(h, P, st);
  if (!P.exec) {
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = run_steps(h, P, h->cap_stream);
    if (rc != PSELINV_OK) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(h->cap_stream, &junk);
      if (junk) cudaGraphDestroy(junk);
      (void)cudaGetLastError();
      return rc;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return cuda_status(e);
    }
    P.graph = g;
    // launches keep the priority of the stream they were captured from
    CK(cudaGraphInstantiate(&P.exec, g, cudaGraphInstantiateFlagUseNodePriority));
  }
  CK(cudaGraphLaunch(P.exec, st));
  return PSELINV_OK;
}

void free_numeric(pselinv_ctx* h) {
  h->factor_plan.release();
  for (auto& pp : h->selinv_plan)
    for (auto& p : pp) p.release();
  cudaFree(h->lu);
  cudaFree(h->nf);
  cudaFree(h->ainv);
  cudaFree(h->scratch);
  cudaFree(h->staging);
  cudaFree(h->outstage);
  cudaFree(h->cbuf);
  cudaFree(h->rcmax);
  h->lu = h->nf = h->ainv = h->scratch = h->staging = h->outstage = h->cbuf = nullptr;
  h->rcmax = nullptr;
  h->dtype = 0;
  h->nbatch = 0;
  h->factored = h->inverted = false;
}

// Common tail of the analyses: widest supernode, the input pattern (for
// the consumers), and the device copy of the structure.
int finish_analyze(pselinv_ctx* h, int64_t n, const int64_t* colptr, const int64_t* rowind,
                   pselinv_t* out) {
  for (int64_t k = 0; k < h->H.ns; k++) h->max_width = std::max<int>(h->max_width, (int)h->H.sn_width[k]);
  h->colptr_h.assign(colptr, colptr + n + 1);
  h->rowind_h.assign(rowind, rowind + colptr[n]);
  if (!h->opts.host_only) {
    if (cudaGetDevice(&h->device) != cudaSuccess) {
      (void)cudaGetLastError();
      delete h;
      return PSELINV_ERR_CUDA;
    }
    const int rc = upload_structure(h);
    if (rc != PSELINV_OK) {
      pselinv_free(h);
      return rc;
    }
  }
  *out = h;
  return PSELINV_OK;
}

int read_device_error(pselinv_ctx* h, cudaStream_t st) {
  int herr[2] = {0, 0};
  CK(cudaMemcpyAsync(herr, h->derr, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (herr[0] == DEV_ZERO_PIVOT) {
    h->last_info = herr[1];
    return PSELINV_ERR_ZERO_PIVOT;
  }
  if (herr[0] == DEV_CHECK) {
    h->last_info = herr[1];
    return PSELINV_ERR_CHECK;
  }
  if (herr[0] == DEV_TIMEOUT) return PSELINV_ERR_TIMEOUT;
  return PSELINV_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

void pselinv_default_opts(pselinv_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_supernode = 256;
  o->relax_pct = 20;
  o->precision = PSELINV_PREC_FP64;
  o->slices = 0;
  o->schedule = PSELINV_SCHED_LEVEL;
  o->use_graph = 1;
  o->check_level = 0;
  o->host_only = 0;
  o->split_normalise = 0;
  o->symmetric = 0;
  o->factor_precision = PSELINV_PREC_FP64;
  o->factor_split_mflops = 0;
}

const char* pselinv_error_string(int status) {
  switch (status) {
    case PSELINV_OK: return "ok";
    case PSELINV_ERR_ARG: return "invalid argument or call order";
    case PSELINV_ERR_NOT_STRUCT_SYM: return "pattern is not structurally symmetric";
    case PSELINV_ERR_ZERO_PIVOT: return "zero pivot in the LU factorisation";
    case PSELINV_ERR_OOM: return "out of memory";
    case PSELINV_ERR_CUDA: return "CUDA error";
    case PSELINV_ERR_TIMEOUT: return "bounded device wait timed out";
    case PSELINV_ERR_CHECK: return "index map read out of range";
    case PSELINV_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
  }
}

int pselinv_analyze(int64_t n, const int64_t* colptr, const int64_t* rowind, const int64_t* perm,
                    const pselinv_opts* opts, pselinv_t* out) {
  if (!out) return PSELINV_ERR_ARG;
  *out = nullptr;
  pselinv_ctx* h = new (std::nothrow) pselinv_ctx();
  if (!h) return PSELINV_ERR_OOM;
  if (opts) h->opts = *opts; else pselinv_default_opts(&h->opts);
  if (h->opts.max_supernode < 1 || h->opts.max_supernode > 256 || h->opts.nd_leaf < 0 ||
      (h->opts.factor_precision != PSELINV_PREC_FP64 &&
       h->opts.factor_precision != PSELINV_PREC_OZAKI_FP16)) {
    delete h;
    return PSELINV_ERR_ARG;
  }
  std::vector<int64_t> nd;  // the nested-dissection ordering asked for by opts.nd_leaf
  if (!perm && h->opts.nd_leaf > 0 && n > 0) {
    try {
      nd.resize((size_t)n);
    } catch (const std::bad_alloc&) {
      delete h;
      return PSELINV_ERR_OOM;
    }
    const int orc = pselinv_order_nd(n, colptr, rowind, h->opts.nd_leaf, nd.data());
    if (orc != PSELINV_OK) {
      delete h;
      return orc;
    }
    perm = nd.data();
  }
  const int rc = analyze_host(n, colptr, rowind, perm, h->opts.max_supernode, h->opts.relax_pct,
                              h->H);
  if (rc != PSELINV_OK) {
    delete h;
    return rc;
  }
  return finish_analyze(h, n, colptr, rowind, out);
}

int pselinv_analyze_general(int64_t n, const int64_t* colptr, const int64_t* rowind,
                            const int64_t* rperm, const int64_t* cperm, const pselinv_opts* opts,
                            pselinv_t* out) {
  if (!out) return PSELINV_ERR_ARG;
  *out = nullptr;
  pselinv_ctx* h = new (std::nothrow) pselinv_ctx();
  if (!h) return PSELINV_ERR_OOM;
  if (opts) h->opts = *opts; else pselinv_default_opts(&h->opts);
  if (h->opts.max_supernode < 1 || h->opts.max_supernode > 256 || h->opts.symmetric ||
      (h->opts.factor_precision != PSELINV_PREC_FP64 &&
       h->opts.factor_precision != PSELINV_PREC_OZAKI_FP16)) {
    delete h;
    return PSELINV_ERR_ARG;
  }
  const int rc = analyze_general_host(n, colptr, rowind, rperm, cperm, h->opts.max_supernode,
                                      h->opts.relax_pct, h->H);
  if (rc != PSELINV_OK) {
    delete h;
    return rc;
  }
  return finish_analyze(h, n, colptr, rowind, out);
}

int pselinv_group(const pselinv_t* members, int64_t count, const pselinv_opts* opts,
                  pselinv_t* out) {
  if (!out) return PSELINV_ERR_ARG;
  *out = nullptr;
  if (!members || count < 1) return PSELINV_ERR_ARG;
  int64_t N = 0, NNZ = 0;
  for (int64_t m = 0; m < count; m++) {
    if (!members[m]) return PSELINV_ERR_ARG;
    if (members[m]->H.general) return PSELINV_ERR_UNSUPPORTED;
    N += members[m]->H.n;
    NNZ += (int64_t)members[m]->rowind_h.size();
  }
  std::vector<int64_t> colptr, rowind, perm;
  try {
    colptr.reserve((size_t)N + 1);
    rowind.reserve((size_t)NNZ);
    perm.reserve((size_t)N);
  } catch (const std::bad_alloc&) {
    return PSELINV_ERR_OOM;
  }
  // direct sum A_1 (+) A_2 (+) ...: member m's rows and columns shifted by
  // the sizes before it, its ordering likewise (block diagonal, so the
  // elimination forest is the union of the members' trees)
  colptr.push_back(0);
  int64_t roff = 0, zoff = 0;
  for (int64_t m = 0; m < count; m++) {
    const pselinv_ctx* g = members[m];
    const int64_t n = g->H.n;
    for (int64_t j = 0; j < n; j++) colptr.push_back(zoff + g->colptr_h[(size_t)j + 1]);
    for (int64_t r : g->rowind_h) rowind.push_back(r + roff);
    for (int64_t j = 0; j < n; j++) perm.push_back(g->H.perm[(size_t)j] + roff);
    roff += n;
    zoff += (int64_t)g->rowind_h.size();
  }
  pselinv_opts o = opts ? *opts : members[0]->opts;
  if (!opts) o.host_only = 0;
  for (int64_t m = 0; m < count && !opts; m++)
    if (!members[m]->opts.host_only) o.host_only = 0;
  return pselinv_analyze(N, colptr.data(), rowind.data(), perm.data(), &o, out);
}

int pselinv_factor(pselinv_t h, int dtype, int64_t nbatch, const void* values, void* stream) {
  if (!h || h->opts.host_only || (dtype != PSELINV_F64 && dtype != PSELINV_C128) || nbatch < 1 ||
      (!values && h->H.nnz > 0))
    return PSELINV_ERR_ARG;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = dtype == PSELINV_F64 ? 8 : 16;
  if (h->dtype != dtype || h->nbatch != nbatch) {
    free_numeric(h);
    h->dtype = dtype;
    h->nbatch = nbatch;
    h->esize = es;
    const size_t sbytes = (size_t)nbatch * h->H.storage * es + 256;
    CK(cudaMalloc(&h->lu, sbytes));
    CK(cudaMalloc(&h->nf, sbytes));
    CK(cudaMalloc(&h->ainv, sbytes));
    CK(cudaMemset(h->nf, 0, sbytes));
    h->scratch_bytes = scratch_need(h->H, nbatch, es);
    CK(cudaMalloc(&h->scratch, h->scratch_bytes));
    CK(cudaMalloc(&h->staging, (size_t)nbatch * h->H.nnz * es + 256));
    CK(cudaMalloc(&h->outstage, (size_t)h->H.nnz * es + 256));
    CK(cudaMalloc(&h->rcmax, (size_t)nbatch * 2 * h->H.n * 8 + 256));
    CK(prepare_dense_kernels(dtype, h->max_width));
    CK(prepare_map_kernels());
    CK(prepare_ozaki_kernels());
    h->slices = h->opts.slices <= 0 ? 6 : std::min(6, std::max(4, (int)h->opts.slices));
  }
  if (!h->factor_plan.built) {
    const int rc = build_factor_plan(h);
    if (rc != PSELINV_OK) return rc;
  }
  h->factored = h->inverted = false;
  if (h->H.nnz > 0)
    CK(cudaMemcpyAsync(h->staging, values, (size_t)nbatch * h->H.nnz * es, cudaMemcpyDefault, st));
  CK(cudaMemsetAsync(h->derr, 0, 4 * sizeof(int), st));
  int rc = run_plan(h, h->factor_plan, st, h->opts.use_graph != 0);
  if (rc != PSELINV_OK) return rc;
  rc = read_device_error(h, st);
  if (rc != PSELINV_OK) return rc;
  h->factored = true;
  return PSELINV_OK;
}

int pselinv_selinv(pselinv_t h, int precision, void* stream) {
  if (!h || !h->factored) return PSELINV_ERR_ARG;
  if (precision < 0) precision = h->opts.precision;
  if (precision != PSELINV_PREC_FP64 && precision != PSELINV_PREC_OZAKI_FP16) return PSELINV_ERR_ARG;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int sched = h->opts.schedule == PSELINV_SCHED_PER_SUPERNODE ? 1 : 0;
  Plan& P = h->selinv_plan[precision][sched];
  if (!P.built) {
    const int rc = build_selinv_plan(h, sched, precision);
    if (rc != PSELINV_OK) return rc;
  }
  h->last_precision = precision;
  const int rc = run_plan(h, P, st, h->opts.use_graph != 0);
  if (rc != PSELINV_OK) return rc;
  h->inverted = true;
  return PSELINV_OK;
}

int pselinv_partition(pselinv_t h, int32_t nranks, int32_t* owner) {
  if (!h || nranks < 1 || !owner) return PSELINV_ERR_ARG;
  const HostSym& H = h->H;
  if (H.general) return PSELINV_ERR_UNSUPPORTED;
  const int64_t ns = H.ns;
  // flops of every supernode and of the subtree below it (children first)
  std::vector<double> f(ns), F(ns, 0.0);
  std::vector<std::vector<int64_t>> children(ns);
  for (int64_t k = 0; k < ns; k++) {
    const double s = (double)H.sn_width[k], c = (double)cK(H, k);
    f[k] = 4 * c * c * s + 4 * c * s * s + 4.0 / 3.0 * s * s * s;
    if (H.sn_parent[k] >= 0) children[H.sn_parent[k]].push_back(k);
  }
  for (int64_t k = 0; k < ns; k++) {  // parents have larger indices
    F[k] += f[k];
    if (H.sn_parent[k] >= 0) F[H.sn_parent[k]] += F[k];
  }
  // split the heaviest subtree of the frontier into its children until the
  // frontier has about eight subtrees per rank or the heaviest one is
  // small against the share of a rank; the split roots form the top part
  std::vector<int64_t> frontier;
  for (int64_t k = 0; k < ns; k++) {
    owner[k] = -1;
    if (H.sn_parent[k] < 0) frontier.push_back(k);
  }
  double total = 0;
  for (int64_t r : frontier) total += F[r];
  if (nranks > 1)
    for (;;) {
      size_t best = frontier.size();
      for (size_t i = 0; i < frontier.size(); i++)
        if (!children[frontier[i]].empty() &&
            (best == frontier.size() || F[frontier[i]] > F[frontier[best]]))
          best = i;
      if (best == frontier.size()) break;
      const int64_t r = frontier[best];
      if ((int64_t)frontier.size() >= 8 * (int64_t)nranks && F[r] <= total / (4.0 * nranks)) break;
      frontier.erase(frontier.begin() + (std::ptrdiff_t)best);
      for (int64_t c : children[r]) frontier.push_back(c);
    }
  // longest processing time first: heaviest subtree to the least loaded rank
  std::sort(frontier.begin(), frontier.end(), [&](int64_t a, int64_t b) { return F[a] > F[b]; });
  std::vector<double> load((size_t)nranks, 0.0);
  std::vector<int32_t> root_rank(ns, -1);
  for (int64_t r : frontier) {
    const int32_t q = (int32_t)(std::min_element(load.begin(), load.end()) - load.begin());
    load[(size_t)q] += F[r];
    root_rank[r] = q;
  }
  // every supernode below a frontier root belongs to that root's rank
  for (int64_t k = ns - 1; k >= 0; k--) {
    if (root_rank[k] >= 0) owner[k] = root_rank[k];
    else if (H.sn_parent[k] >= 0 && owner[H.sn_parent[k]] >= 0) owner[k] = owner[H.sn_parent[k]];
  }
  return PSELINV_OK;
}

int pselinv_set_subset(pselinv_t h, const int32_t* owner, int32_t rank) {
  if (!h) return PSELINV_ERR_ARG;
  if (owner && h->H.general) return PSELINV_ERR_UNSUPPORTED;
  if (owner) {
    h->subset.assign((size_t)h->H.ns, 0);
    for (int64_t k = 0; k < h->H.ns; k++) h->subset[(size_t)k] = owner[k] == rank ? 1 : 0;
  } else {
    h->subset.clear();
  }
  for (auto& pp : h->selinv_plan)
    for (auto& p : pp) p.release();
  return PSELINV_OK;
}

// G_K = Ainv(R_K, R_K) of instance `batch` between `buf` (device, c x c
// column-major) and the handle's storage: export gathers it, import writes
// it back into the ancestors' blocks it comes from.
static int block_transfer(pselinv_t h, int64_t K, int64_t batch, void* buf, bool import,
                          cudaStream_t st) {
  if (!h || !h->factored || K < 0 || K >= h->H.ns || batch < 0 || batch >= h->nbatch || !buf)
    return PSELINV_ERR_ARG;
  if (h->H.general) return PSELINV_ERR_UNSUPPORTED;
  if (!is_device_ptr(buf)) return PSELINV_ERR_ARG;
  const int64_t c = cK(h->H, K);
  if (c == 0) return PSELINV_OK;
  CK(cudaSetDevice(h->device));
  std::vector<SnTask> tasks;
  for (int tq = 0; tq < ceil_div(c, 32); tq++)
    for (int tp = 0; tp < ceil_div(c, 32); tp++) tasks.push_back({(int)batch, (int)K, tp, tq});
  const size_t tb = align256(tasks.size() * sizeof(SnTask)), ob = align256(tasks.size() * 8);
  if (tb + ob > h->blk_buf_bytes) {
    CK(cudaStreamSynchronize(st));
    if (h->blk_buf) cudaFree(h->blk_buf);
    h->blk_buf = nullptr;
    h->blk_buf_bytes = 0;
    CK(cudaMalloc(&h->blk_buf, tb + ob));
    h->blk_buf_bytes = tb + ob;
  }
  char* d = (char*)h->blk_buf;
  CK(cudaMemcpyAsync(d, tasks.data(), tasks.size() * sizeof(SnTask), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(d + tb, 0, tasks.size() * 8, st));
  if (import)
    launch_scatter_set(h->dtype, h->S, h->ainv, buf, (const int64_t*)(d + tb),
                       (const SnTask*)d, (int)tasks.size(), st);
  else
    launch_gather(h->dtype, h->S, h->ainv, buf, (const int64_t*)(d + tb), (const SnTask*)d,
                  (int)tasks.size(), st);
  CK(cudaGetLastError());
  // the host task list must outlive the copy
  CK(cudaStreamSynchronize(st));
  return PSELINV_OK;
}

int pselinv_export_block(pselinv_t h, int64_t K, int64_t batch, void* out, void* stream) {
  return block_transfer(h, K, batch, out, false, (cudaStream_t)stream);
}

int pselinv_import_block(pselinv_t h, int64_t K, int64_t batch, const void* in, void* stream) {
  const int rc = block_transfer(h, K, batch, const_cast<void*>(in), true, (cudaStream_t)stream);
  if (rc == PSELINV_OK && h) h->inverted = true;
  return rc;
}

int pselinv_set_factor_precision(pselinv_t h, int precision, int32_t split_mflops) {
  if (!h || (precision != PSELINV_PREC_FP64 && precision != PSELINV_PREC_OZAKI_FP16))
    return PSELINV_ERR_ARG;
  h->opts.factor_precision = precision;
  h->opts.factor_split_mflops = split_mflops;
  h->factor_plan.release();
  return PSELINV_OK;
}

int pselinv_set_schedule(pselinv_t h, int schedule) {
  if (!h || (schedule != PSELINV_SCHED_LEVEL && schedule != PSELINV_SCHED_PER_SUPERNODE))
    return PSELINV_ERR_ARG;
  h->opts.schedule = schedule;
  return PSELINV_OK;
}

int pselinv_get_selected(pselinv_t h, int layout, int64_t batch, void* out, void* stream) {
  if (!h || !out || batch < 0 || batch >= h->nbatch) return PSELINV_ERR_ARG;
  if (layout == PSELINV_LAYOUT_FACTORS ? !h->factored : !h->inverted) return PSELINV_ERR_ARG;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = is_device_ptr(out);
  if (layout == PSELINV_LAYOUT_FACTORS) {
    CK(cudaMemcpyAsync(out, h->lu + (size_t)batch * h->H.storage * h->esize,
                       (size_t)h->H.storage * h->esize, cudaMemcpyDefault, st));
    if (!dev) CK(cudaStreamSynchronize(st));
    return PSELINV_OK;
  }
  if (layout == PSELINV_LAYOUT_PATTERN_A) {
    void* dst = dev ? out : (void*)h->outstage;
    launch_extract(h->dtype, h->S, h->ainv, (int)batch, dst, st);
    CK(cudaGetLastError());
    if (!dev) {
      CK(cudaMemcpyAsync(out, h->outstage, (size_t)h->H.nnz * h->esize, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    return PSELINV_OK;
  }
  if (layout == PSELINV_LAYOUT_SUPERNODAL) {
    CK(cudaMemcpyAsync(out, h->ainv + (size_t)batch * h->H.storage * h->esize,
                       (size_t)h->H.storage * h->esize, cudaMemcpyDefault, st));
    if (!dev) CK(cudaStreamSynchronize(st));
    return PSELINV_OK;
  }
  return PSELINV_ERR_ARG;
}

int pselinv_get_structure(pselinv_t h, pselinv_structure* o) {
  if (!h || !o) return PSELINV_ERR_ARG;
  const HostSym& H = h->H;
  o->n = H.n;
  o->nsuper = H.ns;
  o->nlevels = (int64_t)H.level_ptr.size() - 1;
  o->storage_size = H.storage;
  o->nnz_a = H.nnz;
  o->perm = H.perm.data();
  o->etree = H.etree.data();
  o->sn_first = H.sn_first.data();
  o->sn_width = H.sn_width.data();
  o->sn_parent = H.sn_parent.data();
  o->sn_depth = H.sn_depth.data();
  o->sn_offset = H.sn_offset.data();
  o->rows_ptr = H.rows_ptr.data();
  o->rows = H.rows.data();
  o->level_ptr = H.level_ptr.data();
  o->level_sn = H.level_sn.data();
  o->value_map = H.value_map.data();
  o->flops_selinv = H.flops_selinv;
  o->flops_selinv_exact = H.flops_selinv_exact;
  o->flops_factor = H.flops_factor;
  o->general = H.general ? 1 : 0;
  o->rperm = H.general ? H.rperm.data() : H.perm.data();
  o->urows_ptr = H.general ? H.urows_ptr.data() : H.rows_ptr.data();
  o->urows = H.general ? H.urows.data() : H.rows.data();
  o->out_map = H.general ? H.inv_map.data() : H.value_map.data();
  return PSELINV_OK;
}

int pselinv_profile(pselinv_t h, int which, void* stream, pselinv_step_stat* out, int64_t cap,
                    int64_t* count) {
  if (!h || which < 0 || which > 2 || !count || (cap > 0 && !out)) return PSELINV_ERR_ARG;
  if (which != 1 ? !h->factored : h->nbatch == 0) return PSELINV_ERR_ARG;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int sched = h->opts.schedule == PSELINV_SCHED_PER_SUPERNODE ? 1 : 0;
  const int prec = h->last_precision;
  if (which != 1 && !h->selinv_plan[prec][sched].built) {
    const int rc = build_selinv_plan(h, sched, prec);
    if (rc != PSELINV_OK) return rc;
  }
  Plan& P = which != 1 ? h->selinv_plan[prec][sched] : h->factor_plan;
  const size_t ns = P.steps.size();
  // which 0/1: serialised, ev[i] .. ev[i + 1] around launch i;
  // which 2: the plan's own streams, ev[2i + 1] before and ev[2i + 2] after
  //   launch i on its stream, ev[0] at the start
  std::vector<cudaEvent_t> ev(which == 2 ? 2 * ns + 1 : ns + 1);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  CK(cudaEventRecord(ev[0], st));
  if (which == 2 && P.two_streams) {
    SweepStreams q3;
    const int rc = sweep_streams(h, &q3);
    if (rc != PSELINV_OK) return rc;
    CK(cudaStreamWaitEvent(q3.main, ev[0], 0));
    CK(cudaStreamWaitEvent(q3.side, ev[0], 0));
    CK(cudaStreamWaitEvent(q3.third, ev[0], 0));
    for (size_t i = 0; i < ns; i++) {
      const Step& s = P.steps[i];
      cudaStream_t q = s.side == 1 ? q3.side : s.side == 2 ? q3.third : q3.main;
      if (s.wait >= 0) CK(cudaStreamWaitEvent(q, P.ev[s.wait], 0));
      CK(cudaEventRecord(ev[2 * i + 1], q));
      launch_step(h, P, s, q);
      CK(cudaEventRecord(ev[2 * i + 2], q));
      if (s.signal >= 0) CK(cudaEventRecord(P.ev[s.signal], q));
    }
    CK(cudaEventRecord(P.ev[EV_MAIN_JOIN], q3.main));
    CK(cudaEventRecord(P.ev[EV_SIDE_JOIN], q3.side));
    CK(cudaEventRecord(P.ev[EV_THIRD_JOIN], q3.third));
    CK(cudaStreamWaitEvent(st, P.ev[EV_MAIN_JOIN], 0));
    CK(cudaStreamWaitEvent(st, P.ev[EV_SIDE_JOIN], 0));
    CK(cudaStreamWaitEvent(st, P.ev[EV_THIRD_JOIN], 0));
  } else if (which == 2) {
    for (size_t i = 0; i < ns; i++) {
      CK(cudaEventRecord(ev[2 * i + 1], st));
      launch_step(h, P, P.steps[i], st);
      CK(cudaEventRecord(ev[2 * i + 2], st));
    }
  } else {
    for (size_t i = 0; i < ns; i++) {
      launch_step(h, P, P.steps[i], st);
      CK(cudaEventRecord(ev[i + 1], st));
    }
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  *count = (int64_t)ns;
  for (size_t i = 0; i < ns && (int64_t)i < cap; i++) {
    float ms = 0, t0 = 0;
    if (which == 2) {
      CK(cudaEventElapsedTime(&t0, ev[0], ev[2 * i + 1]));
      CK(cudaEventElapsedTime(&ms, ev[2 * i + 1], ev[2 * i + 2]));
    } else {
      CK(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
    }
    out[i].start_ms = t0;
    const Step& s = P.steps[i];
    static const int kinds[] = {PSELINV_STEP_GEMM,    PSELINV_STEP_TRI_INV,
                                PSELINV_STEP_GATHER,  PSELINV_STEP_SCATTER_SUB, PSELINV_STEP_COPY,
                                PSELINV_STEP_MEMSET,  PSELINV_STEP_SCATTER_VALUES,
                                PSELINV_STEP_SLICE,   PSELINV_STEP_OZAKI_GEMM, PSELINV_STEP_MEMSET,
                                PSELINV_STEP_DIAG_LU, PSELINV_STEP_SMALL_LEVEL,
                                PSELINV_STEP_GATHER_SLICE, PSELINV_STEP_OUTPUT_MAXIMA,
                                PSELINV_STEP_COPY};
    out[i].kind = kinds[s.kind];
    out[i].level = s.level;
    out[i].tasks = s.n;
    out[i].flops = s.flops;
    out[i].bytes = (double)s.bytes;
    out[i].ms = ms;
    out[i].param = (s.kind == ST_GEMM || s.kind == ST_OZGEMM) ? s.param
                   : s.kind == ST_TRI_INV                  ? s.cfg
                                                           : -1;
    out[i].side = s.side;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (which != 1) h->inverted = true;
  return read_device_error(h, st);
}

int pselinv_plan_stats(pselinv_t h, int64_t* launches_selinv, int64_t* launches_factor) {
  if (!h) return PSELINV_ERR_ARG;
  const int sched = h->opts.schedule == PSELINV_SCHED_PER_SUPERNODE ? 1 : 0;
  const Plan& sp = h->selinv_plan[h->last_precision][sched];
  auto kernels = [](const Plan& P) -> int64_t {
    if (!P.built) return 0;
    int64_t n = 0;
    for (const Step& s : P.steps) n += s.kind != ST_MEMSET;
    return n;
  };
  if (launches_selinv) *launches_selinv = kernels(sp);
  if (launches_factor) *launches_factor = kernels(h->factor_plan);
  return PSELINV_OK;
}

}  // extern "C"

// Cost-model tuning: predict the time of every candidate of every tunable
// launch with the model and keep the argmin (no timing).
template <class RB>
static int model_tune(pselinv_ctx* h, Plan& P0, int precision, pselinv_model_t model, RB rebuild) {
  if (!model) return PSELINV_ERR_ARG;
  static const int gemm_cands[4] = {GEMM_64x64, GEMM_32x32, GEMM_128x64, GEMM_ROWS};
  constexpr double kTuneFp64MaxFlops = 2e10;
  static const int ks_cands[5] = {1, 2, 4, 8, 16};
  std::vector<std::tuple<int, int, int>> keys;
  std::vector<pselinv_tune_record> q;
  for (const Step& s : P0.steps) {
    if (s.slot < 0) continue;
    const auto key = std::make_tuple(s.level, s.slot, (int)s.kind);
    if (std::find(keys.begin(), keys.end(), key) != keys.end()) continue;
    keys.push_back(key);
    const int nc = s.kind == ST_GEMM ? 4 : 5;
    for (int v = 0; v < nc; v++) {
      pselinv_tune_record r{};
      r.precision = precision;
      r.level = s.level;
      r.slot = s.slot;
      r.kind = s.kind == ST_GEMM ? PSELINV_STEP_GEMM : PSELINV_STEP_OZAKI_GEMM;
      r.param = s.kind == ST_GEMM ? gemm_cands[v] : ks_cands[v];
      for (int i = 0; i < 8; i++) r.feat[i] = s.feat[i];
      q.push_back(r);
    }
  }
  std::vector<double> pred(q.size());
  int rc = pselinv_model_predict(model, q.data(), (int64_t)q.size(), pred.data(), nullptr);
  if (rc != PSELINV_OK) return rc;
  for (const auto& key : keys) {
    double bp = 1e300;
    int best = -1;
    for (size_t i = 0; i < q.size(); i++)
      if (q[i].level == std::get<0>(key) && q[i].slot == std::get<1>(key) && pred[i] < bp) {
        bp = pred[i];
        best = q[i].param;
      }
    if (best >= 0) h->tuned[std::make_tuple(precision, std::get<0>(key), std::get<1>(key))] = best;
  }
  return rebuild();
}

template <class RB>
static int model_tune(pselinv_ctx* h, Plan& P0, int precision, pselinv_model_t model, RB rebuild);

extern "C" {

int pselinv_tune(pselinv_t h, int precision, int mode, pselinv_model_t model, void* stream) {
  if (!h || !h->factored || (precision != PSELINV_PREC_FP64 && precision != PSELINV_PREC_OZAKI_FP16))
    return PSELINV_ERR_ARG;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int sched = h->opts.schedule == PSELINV_SCHED_PER_SUPERNODE ? 1 : 0;
  auto rebuild = [&]() -> int {
    for (auto& p : h->selinv_plan[precision]) p.release();
    return build_selinv_plan(h, sched, precision);
  };
  // drop this precision's tuned values
  for (auto it = h->tuned.begin(); it != h->tuned.end();)
    it = std::get<0>(it->first) == precision ? h->tuned.erase(it) : std::next(it);
  int rc = rebuild();
  if (rc != PSELINV_OK || mode == PSELINV_TUNE_RESET) return rc;
  Plan& P0 = h->selinv_plan[precision][sched];
  if (mode == PSELINV_TUNE_MODEL) return model_tune(h, P0, precision, model, rebuild);
  if (mode != PSELINV_TUNE_EXHAUSTIVE) return PSELINV_ERR_ARG;

  static const int gemm_cands[4] = {GEMM_64x64, GEMM_32x32, GEMM_128x64, GEMM_ROWS};
  constexpr double kTuneFp64MaxFlops = 2e10;
  static const int ks_cands[5] = {1, 2, 4, 8, 16};
  struct Key {
    int level, slot, kind;
  };
  std::vector<Key> keys;
  std::map<std::tuple<int, int, int>, std::vector<float>> feats;
  for (const Step& s : P0.steps)
    if (s.slot >= 0) {
      const auto k = std::make_tuple(s.level, s.slot, (int)s.kind);
      if (!feats.count(k)) {
        keys.push_back({s.level, s.slot, (int)s.kind});
        feats[k] = std::vector<float>(s.feat, s.feat + 8);
      }
    }
  std::map<std::tuple<int, int, int, int>, double> best_ms;  // (level, slot, kind, value) -> ms
  std::map<std::pair<int, int>, double> level_ms;  // (level, mode) -> ms of its launches
  std::vector<pselinv_step_stat> stats;
  auto measure = [&](int mode_tag) -> int {
    int r = rebuild();
    if (r != PSELINV_OK) return r;
    h->last_precision = precision;
    Plan& P = h->selinv_plan[precision][sched];
    for (const Step& s : P.steps)
      if (s.slot >= 0) {
        const auto k = std::make_tuple(s.level, s.slot, (int)s.kind);
        if (!feats.count(k)) {
          keys.push_back({s.level, s.slot, (int)s.kind});
          feats[k] = std::vector<float>(s.feat, s.feat + 8);
        }
      }
    for (int rep = 0; rep < 2; rep++) {
      stats.assign(P.steps.size(), pselinv_step_stat{});
      int64_t cnt = 0;
      r = pselinv_profile(h, 0, stream, stats.data(), (int64_t)stats.size(), &cnt);
      if (r != PSELINV_OK) return r;
      std::map<std::tuple<int, int, int, int>, double> acc;
      std::map<int, double> lev_acc;
      for (size_t i = 0; i < P.steps.size(); i++) {
        const Step& s = P.steps[i];
        if (s.level >= 0) lev_acc[s.level] += stats[i].ms;
        if (s.slot < 0) continue;
        // phase B keeps its large levels split at their default K split,
        // which need not be a candidate: only phase A times K splits
        if (mode_tag == 1 && s.kind == ST_OZGEMM) continue;
        acc[std::make_tuple(s.level, s.slot, (int)s.kind, s.param)] += stats[i].ms;
      }
      for (const auto& kv : acc) {
        auto it = best_ms.find(kv.first);
        if (it == best_ms.end() || kv.second < it->second) best_ms[kv.first] = kv.second;
      }
      if (mode_tag >= 0)
        for (const auto& kv : lev_acc) {
          const auto k = std::make_pair(kv.first, mode_tag);
          auto it = level_ms.find(k);
          if (it == level_ms.end() || kv.second < it->second) level_ms[k] = kv.second;
        }
    }
    return PSELINV_OK;
  };
  const int nlev = (int)h->H.level_ptr.size() - 1;
  if (precision == PSELINV_PREC_FP64) {
    for (int v = 0; v < 4; v++) {
      for (const Key& k : keys) h->tuned[std::make_tuple(precision, k.level, k.slot)] = gemm_cands[v];
      rc = measure(-1);
      if (rc != PSELINV_OK) return rc;
    }
  } else {
    // phase A: every level split, K splits 1..16
    for (int v = 0; v < 5; v++) {
      for (int l = 0; l < nlev; l++) {
        h->tuned[std::make_tuple(precision, l, 3)] = 0;
        h->tuned[std::make_tuple(precision, l, 1)] = ks_cands[v];
        h->tuned[std::make_tuple(precision, l, 2)] = ks_cands[v];
        h->tuned[std::make_tuple(precision, l, 0)] = gemm_cands[(v + 3) % 4];
      }
      rc = measure(0);
      if (rc != PSELINV_OK) return rc;
    }
    // phase B: FP64 levels, tile shapes and row panels.  Only levels whose
    // products are small enough that FP64 could win are run in FP64 (a level
    // of kTuneFp64MaxFlops takes about 20 ms in FP64 and 1 ms split); the
    // others stay split at the default K split and keep that mode.
    for (int v = 0; v < 4; v++) {
      for (int l = 0; l < nlev; l++) {
        if (level_product_flops(h, l) > kTuneFp64MaxFlops) {
          h->tuned.erase(std::make_tuple(precision, l, 1));
          h->tuned.erase(std::make_tuple(precision, l, 2));
          h->tuned[std::make_tuple(precision, l, 3)] = 0;
          continue;
        }
        h->tuned[std::make_tuple(precision, l, 3)] = 1;
        h->tuned[std::make_tuple(precision, l, 4)] = gemm_cands[v];
        h->tuned[std::make_tuple(precision, l, 5)] = gemm_cands[v];
      }
      rc = measure(1);
      if (rc != PSELINV_OK) return rc;
    }
    h->tuned.clear();
  }
  // keep the fastest candidate of every tunable launch; record everything
  h->records.clear();
  for (const Key& k : keys) {
    int best = -1;
    double bms = 1e300;
    for (const auto& kv : best_ms) {
      if (std::get<0>(kv.first) != k.level || std::get<1>(kv.first) != k.slot ||
          std::get<2>(kv.first) != k.kind)
        continue;
      if (kv.second < bms) {
        bms = kv.second;
        best = std::get<3>(kv.first);
      }
    }
    if (best < 0) continue;
    h->tuned[std::make_tuple(precision, k.level, k.slot)] = best;
    for (const auto& kv : best_ms) {
      if (std::get<0>(kv.first) != k.level || std::get<1>(kv.first) != k.slot ||
          std::get<2>(kv.first) != k.kind)
        continue;
      pselinv_tune_record r{};
      r.precision = precision;
      r.level = k.level;
      r.slot = k.slot;
      r.kind = k.kind == ST_GEMM ? PSELINV_STEP_GEMM : PSELINV_STEP_OZAKI_GEMM;
      r.param = std::get<3>(kv.first);
      r.chosen = r.param == best ? 1 : 0;
      const auto& f = feats[std::make_tuple(k.level, k.slot, k.kind)];
      for (int i = 0; i < 8; i++) r.feat[i] = f[i];
      r.ms = kv.second;
      h->records.push_back(r);
    }
  }
  if (precision == PSELINV_PREC_OZAKI_FP16)
    for (int l = 0; l < nlev; l++) {
      auto a = level_ms.find(std::make_pair(l, 0)), b = level_ms.find(std::make_pair(l, 1));
      if (a != level_ms.end() && b != level_ms.end() && level_product_flops(h, l) <= kTuneFp64MaxFlops)
        h->tuned[std::make_tuple(precision, l, 3)] = b->second < a->second ? 1 : 0;
    }
  rc = rebuild();
  if (rc != PSELINV_OK) return rc;
  // leave valid results of the tuned plan
  rc = run_plan(h, h->selinv_plan[precision][sched], st, false);
  if (rc != PSELINV_OK) return rc;
  CK(cudaStreamSynchronize(st));
  h->inverted = true;
  return PSELINV_OK;
}

int pselinv_measure_fp64_peak(void* stream, double* tflops, double* ms) {
  if (!tflops) return PSELINV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = fp64_peak_grid(sms);
  double* out = nullptr;
  CK(cudaMalloc(&out, (size_t)grid * 256 * sizeof(double)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int iters = 20000;  // about 80 ms at 1.26 TFLOP/s
  double flops = 0;
  float t = 0;
  if (e == cudaSuccess) {
    launch_fp64_peak(out, grid, iters / 10, st);  // warm-up
    e = cudaEventRecord(e0, st);
  }
  if (e == cudaSuccess) {
    flops = launch_fp64_peak(out, grid, iters, st);
    e = cudaEventRecord(e1, st);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  CK(e);
  if (t <= 0.0f) return PSELINV_ERR_CUDA;
  *tflops = flops / ((double)t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return PSELINV_OK;
}

int pselinv_wait_selftest(void* stream, int64_t budget_us) {
  if (budget_us < 1 || budget_us > 2000000) return PSELINV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int* derr = nullptr;
  CK(cudaMalloc(&derr, 4 * sizeof(int)));
  int herr[2] = {0, 0};
  cudaError_t e = cudaMemsetAsync(derr, 0, 4 * sizeof(int), st);
  if (e == cudaSuccess) {
    launch_wait_selftest(derr, (unsigned long long)budget_us * 1000ull, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(herr, derr, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(derr);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return cuda_status(e);
  }
  return herr[0] == DEV_TIMEOUT ? PSELINV_ERR_TIMEOUT : PSELINV_OK;
}

// weights (host) and, for the trace, B (host or device) into the consumer
// buffer: [weights: nbatch scalars | B: nnz scalars | partial sums | result]
static int consumer_stage(pselinv_ctx* h, const void* weights, const void* B, cudaStream_t st) {
  const size_t es = h->esize, nb = (size_t)h->nbatch, nnz = (size_t)h->H.nnz;
  if (!h->cbuf) CK(cudaMalloc(&h->cbuf, align256(nb * es) + align256(nnz * es) + trace_partial_bytes() + 256));
  CK(cudaMemcpyAsync(h->cbuf, weights, nb * es, cudaMemcpyHostToDevice, st));
  if (B) CK(cudaMemcpyAsync(h->cbuf + align256(nb * es), B, nnz * es, cudaMemcpyDefault, st));
  return PSELINV_OK;
}

int pselinv_weighted_sum(pselinv_t h, const void* weights, void* out, void* stream) {
  if (!h || !weights || !out || !h->inverted) return PSELINV_ERR_ARG;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  int rc = consumer_stage(h, weights, nullptr, st);
  if (rc != PSELINV_OK) return rc;
  const bool dev = is_device_ptr(out);
  void* dst = dev ? out : (void*)h->outstage;
  launch_weighted_sum(h->dtype, h->S, h->ainv, (int)h->nbatch, h->cbuf, dst, st);
  CK(cudaGetLastError());
  if (!dev) {
    CK(cudaMemcpyAsync(out, h->outstage, (size_t)h->H.nnz * h->esize, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return PSELINV_OK;
}

int pselinv_trace(pselinv_t h, const void* weights, const void* B, void* out, void* stream) {
  if (!h || !weights || !B || !out || !h->inverted) return PSELINV_ERR_ARG;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = (int64_t)h->colptr_h.size() - 1, nnz = h->H.nnz;
  if (!h->tslot && h->H.general) {
    // Tr[B A^{-1}] = sum_p B[p] (A^{-1})_{col(p), row(p)}: exactly the
    // selected entry returned for each input entry (Eq. sel_entries)
    CK(cudaMalloc(&h->tslot, (size_t)std::max<int64_t>(nnz, 1) * 8));
    CK(cudaMemcpy(h->tslot, h->H.inv_map.data(), (size_t)nnz * 8, cudaMemcpyHostToDevice));
  }
  if (!h->tslot) {
    // transposed entry of every input entry (the pattern is structurally
    // symmetric), then its storage slot
    std::vector<int64_t> col(nnz), order(nnz), tslot(nnz);
    for (int64_t j = 0; j < n; j++)
      for (int64_t q = h->colptr_h[j]; q < h->colptr_h[j + 1]; q++) col[q] = j;
    for (int64_t q = 0; q < nnz; q++) order[q] = q;
    auto key = [&](int64_t q) { return h->rowind_h[q] * n + col[q]; };  // (i, j) -> row-major
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return key(a) < key(b); });
    for (int64_t q = 0; q < nnz; q++) {
      // entry q = (i, j): find (j, i), i.e. row-major key j * n + i
      const int64_t want = col[q] * n + h->rowind_h[q];
      int64_t lo = 0, hi = nnz;
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (key(order[mid]) < want) lo = mid + 1; else hi = mid;
      }
      if (lo >= nnz || key(order[lo]) != want) return PSELINV_ERR_NOT_STRUCT_SYM;
      tslot[q] = h->H.value_map[order[lo]];
    }
    CK(cudaMalloc(&h->tslot, (size_t)std::max<int64_t>(nnz, 1) * 8));
    CK(cudaMemcpy(h->tslot, tslot.data(), (size_t)nnz * 8, cudaMemcpyHostToDevice));
  }
  int rc = consumer_stage(h, weights, B, st);
  if (rc != PSELINV_OK) return rc;
  const size_t es = h->esize, nb = (size_t)h->nbatch;
  char* bdev = h->cbuf + align256(nb * es);
  char* partial = bdev + align256((size_t)nnz * es);
  char* res = partial + trace_partial_bytes();
  launch_trace(h->dtype, h->S, h->ainv, (int)h->nbatch, h->cbuf, bdev, h->tslot, partial, res, st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, res, es, cudaMemcpyDefault, st));
  if (!is_device_ptr(out)) CK(cudaStreamSynchronize(st));
  return PSELINV_OK;
}

int pselinv_plan_get(pselinv_t h, int precision, int32_t* out, int64_t cap, int64_t* count) {
  if (!h || !count || (cap > 0 && !out) ||
      (precision != PSELINV_PREC_FP64 && precision != PSELINV_PREC_OZAKI_FP16))
    return PSELINV_ERR_ARG;
  int64_t n = 0;
  for (const auto& kv : h->tuned) {
    if (std::get<0>(kv.first) != precision) continue;
    if (n < cap) {
      out[3 * n] = std::get<1>(kv.first);
      out[3 * n + 1] = std::get<2>(kv.first);
      out[3 * n + 2] = kv.second;
    }
    n++;
  }
  *count = n;
  return PSELINV_OK;
}

int pselinv_plan_set(pselinv_t h, int precision, const int32_t* in, int64_t count) {
  if (!h || count < 0 || (count > 0 && !in) ||
      (precision != PSELINV_PREC_FP64 && precision != PSELINV_PREC_OZAKI_FP16))
    return PSELINV_ERR_ARG;
  const int nlev = h->H.level_ptr.empty() ? 0 : (int)h->H.level_ptr.size() - 1;
  std::vector<std::pair<std::tuple<int, int, int>, int>> entries;
  for (int64_t i = 0; i < count; i++) {
    const int lev = in[3 * i], slot = in[3 * i + 1], v = in[3 * i + 2];
    bool ok = lev >= 0 && lev < nlev && slot >= 0 && slot <= 5;
    if (ok && precision == PSELINV_PREC_FP64) ok = slot <= 2 && v >= 0 && v <= 3;
    if (ok && precision == PSELINV_PREC_OZAKI_FP16) {
      if (slot == 1 || slot == 2)
        ok = v == 1 || v == 2 || v == 4 || v == 8 || v == 16;
      else if (slot == 3)
        ok = v == 0 || v == 1;
      else
        ok = v >= 0 && v <= 3;
    }
    if (!ok) return PSELINV_ERR_ARG;
    entries.push_back({std::make_tuple(precision, lev, slot), v});
  }
  for (auto it = h->tuned.begin(); it != h->tuned.end();)
    it = std::get<0>(it->first) == precision ? h->tuned.erase(it) : std::next(it);
  for (const auto& e : entries) h->tuned[e.first] = e.second;
  for (auto& p : h->selinv_plan[precision]) p.release();
  return PSELINV_OK;
}

// Tuning cache file: a header line naming the format, the precision and
// the structure it was tuned on (counts and a 64-bit FNV-1a hash of the
// supernode widths, row-structure sizes and depth levels, so that a plan
// tuned for another matrix with the same counts is refused), then one
// "level slot value" line per tuned value (the triples of pselinv_plan_get).
static unsigned long long structure_hash(const HostSym& H) {
  unsigned long long x = 1469598103934665603ull;
  auto mix = [&](int64_t v) {
    for (int b = 0; b < 8; b++) {
      x ^= (unsigned long long)((uint64_t)v >> (8 * b)) & 0xFFull;
      x *= 1099511628211ull;
    }
  };
  auto mixv = [&](const std::vector<int64_t>& v) {
    mix((int64_t)v.size());
    for (int64_t e : v) mix(e);
  };
  mix(H.n);
  mix(H.ns);
  mixv(H.sn_width);
  mixv(H.rows_ptr);
  mixv(H.level_ptr);
  mixv(H.level_sn);
  return x;
}

int pselinv_plan_save(pselinv_t h, int precision, const char* path) {
  if (!h || !path) return PSELINV_ERR_ARG;
  int64_t count = 0;
  int rc = pselinv_plan_get(h, precision, nullptr, 0, &count);
  if (rc != PSELINV_OK) return rc;
  std::vector<int32_t> t((size_t)(3 * count));
  rc = pselinv_plan_get(h, precision, t.data(), count, &count);
  if (rc != PSELINV_OK) return rc;
  FILE* f = std::fopen(path, "w");
  if (!f) return PSELINV_ERR_ARG;
  const int64_t nlev = h->H.level_ptr.empty() ? 0 : (int64_t)h->H.level_ptr.size() - 1;
  bool ok = std::fprintf(f, "pselinv-plan 2 %d %lld %lld %lld %016llx %lld\n", precision,
                         (long long)h->H.n, (long long)h->H.ns, (long long)nlev,
                         structure_hash(h->H), (long long)count) > 0;
  for (int64_t i = 0; i < count && ok; i++)
    ok = std::fprintf(f, "%d %d %d\n", t[3 * i], t[3 * i + 1], t[3 * i + 2]) > 0;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? PSELINV_OK : PSELINV_ERR_ARG;
}

int pselinv_plan_load(pselinv_t h, int precision, const char* path) {
  if (!h || !path || (precision != PSELINV_PREC_FP64 && precision != PSELINV_PREC_OZAKI_FP16))
    return PSELINV_ERR_ARG;
  FILE* f = std::fopen(path, "r");
  if (!f) return PSELINV_ERR_ARG;
  int version = 0, prec = -1;
  long long n = -1, ns = -1, nlev = -1, count = -1;
  unsigned long long hash = 0;
  const int64_t my_nlev = h->H.level_ptr.empty() ? 0 : (int64_t)h->H.level_ptr.size() - 1;
  bool ok = std::fscanf(f, "pselinv-plan %d %d %lld %lld %lld %llx %lld", &version, &prec, &n,
                        &ns, &nlev, &hash, &count) == 7 &&
            version == 2 && prec == precision && n == h->H.n && ns == h->H.ns && nlev == my_nlev &&
            hash == structure_hash(h->H) && count >= 0 && count <= 64 * (my_nlev + 1);
  std::vector<int32_t> t;
  for (long long i = 0; ok && i < count; i++) {
    int a = 0, b = 0, c = 0;
    ok = std::fscanf(f, "%d %d %d", &a, &b, &c) == 3;
    t.push_back(a);
    t.push_back(b);
    t.push_back(c);
  }
  std::fclose(f);
  if (!ok) return PSELINV_ERR_ARG;
  return pselinv_plan_set(h, precision, t.data(), count);  // validates every triple
}

int pselinv_tune_records(pselinv_t h, pselinv_tune_record* out, int64_t cap, int64_t* count) {
  if (!h || !count || (cap > 0 && !out)) return PSELINV_ERR_ARG;
  *count = (int64_t)h->records.size();
  for (int64_t i = 0; i < *count && i < cap; i++) out[i] = h->records[i];
  return PSELINV_OK;
}

int pselinv_sync(pselinv_t h, void* stream) {
  if (!h || h->opts.host_only) return PSELINV_ERR_ARG;
  CK(cudaSetDevice(h->device));
  return read_device_error(h, (cudaStream_t)stream);
}

int64_t pselinv_last_info(pselinv_t h) { return h ? h->last_info : -1; }

void pselinv_free(pselinv_t h) {
  if (!h) return;
  if (!h->opts.host_only && h->device >= 0) {
    cudaSetDevice(h->device);
    free_numeric(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->main_stream) cudaStreamDestroy(h->main_stream);
    if (h->side_stream) cudaStreamDestroy(h->side_stream);
    if (h->third_stream) cudaStreamDestroy(h->third_stream);
    cudaFree(h->dsym);
    cudaFree(h->derr);
    cudaFree(h->tslot);
    if (h->blk_buf) cudaFree(h->blk_buf);
  }
  delete h;
}

}  // extern "C"
