// Device-side types shared by the CUDA sources: scalar types, the view of
// the symbolic structure the kernels read, task/descriptor records and the
// launch functions implemented in the kernel files.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace pselinv {

// ---------------------------------------------------------------------------
// scalars
// ---------------------------------------------------------------------------
struct cdouble {
  double x, y;
};

__host__ __device__ inline double sc_zero(double) { return 0.0; }
__host__ __device__ inline cdouble sc_zero(cdouble) { return {0.0, 0.0}; }
__host__ __device__ inline double sc_one(double) { return 1.0; }
__host__ __device__ inline cdouble sc_one(cdouble) { return {1.0, 0.0}; }

__device__ __forceinline__ double fma_s(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ cdouble fma_s(cdouble a, cdouble b, cdouble c) {
  return {fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}
__device__ __forceinline__ double mul_s(double a, double b) { return a * b; }
__device__ __forceinline__ cdouble mul_s(cdouble a, cdouble b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__device__ __forceinline__ double sub_s(double a, double b) { return a - b; }
__device__ __forceinline__ cdouble sub_s(cdouble a, cdouble b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ double add_s(double a, double b) { return a + b; }
__device__ __forceinline__ cdouble add_s(cdouble a, cdouble b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ double scale_s(double a, double s) { return a * s; }
__device__ __forceinline__ cdouble scale_s(cdouble a, double s) { return {a.x * s, a.y * s}; }
__device__ __forceinline__ double div_s(double a, double b) { return a / b; }
__device__ __forceinline__ cdouble div_s(cdouble a, cdouble b) {
  // Smith's algorithm for complex division
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, d = b.x + b.y * r;
    return {(a.x + a.y * r) / d, (a.y - a.x * r) / d};
  }
  const double r = b.x / b.y, d = b.y + b.x * r;
  return {(a.x * r + a.y) / d, (a.y * r - a.x) / d};
}
__device__ __forceinline__ bool is_zero(double a) { return a == 0.0; }
__device__ __forceinline__ bool is_zero(cdouble a) { return a.x == 0.0 && a.y == 0.0; }
__device__ __forceinline__ void atomic_add_s(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_s(cdouble* p, cdouble v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

// ---------------------------------------------------------------------------
// structure view (device pointers), passed by value
// ---------------------------------------------------------------------------
struct SymDev {
  const int32_t* sn_first;
  const int32_t* sn_width;
  const int32_t* sn_c;
  const int64_t* sn_off;
  const int64_t* rows_ptr;
  const int32_t* rows_blk;
  const int32_t* blk_sn;
  const int32_t* blk_pb;
  const int64_t* blk_rel;
  const int32_t* relidx;
  const int64_t* value_map;
  int64_t storage;  // scalars per instance
  int64_t nnz;
  int32_t ns;
  int32_t check;    // 1: bounds-check map reads
  int64_t relidx_size;
  int* err;         // [0] status, [1] info
  // slot of the selected entry returned for each input entry (extraction,
  // weighted sums): value_map for structurally symmetric handles
  const int64_t* out_map;
  // Storage bases of the gather of G_K = Ainv(R_U(K), R_L(K)) (R_U = R_L =
  // R_K for structurally symmetric handles), precomputed per position.
  // Column side, position q of R_L(K) (index rows_ptr[K] + q), y = R_L[q]
  // in supernode J = col_sn: Ainv(x, y) for x in J or later lies at
  // (x in J ? col_diag : col_pan)[q] + relidx[col_rel[q] + p], p the
  // position of x in R_U(K).  Row side, position p of R_U(K) (index
  // urows_ptr[K] + p, or rows_ptr[K] + p), x = R_U[p] in supernode I =
  // row_sn: Ainv(x, y) for y after I lies at row_pan[p] + relidx[row_rel[p] + q].
  const int64_t* col_diag;
  const int64_t* col_pan;
  const int64_t* col_rel;
  const int32_t* col_sn;
  const int64_t* row_pan;
  const int64_t* row_rel;
  const int32_t* row_sn;
  // global (permuted) index of every position of R_L(K) / R_K (lrows, all
  // handles) and of R_U(K) (urows, general handles; lrows otherwise)
  const int32_t* lrows;
  const int32_t* urows;
  int64_t n;
  // general patterns (general = 1; null for structurally symmetric
  // handles): sn_c, rows_ptr, rows_blk and blk_* describe R_L(K) (the L
  // panel's rows), sn_cu, urows_ptr, urows_blk and ublk_* R_U(K) (the U^T
  // panel's rows); a block of R_L(K) maps the positions of R_U(K) from
  // blk_q0 on (relidx at blk_rel - blk_q0) and a block of R_U(K) those of
  // R_L(K) from ublk_q0 on; lrows / urows hold R_L and R_U themselves.
  int32_t general;
  const int32_t* sn_cu;
  const int64_t* urows_ptr;
  const int32_t* urows_blk;
  const int32_t* blk_q0;
  const int32_t* ublk_sn;
  const int64_t* ublk_rel;
  const int32_t* ublk_q0;
};

enum DevErr { DEV_OK = 0, DEV_ZERO_PIVOT = 1, DEV_CHECK = 2, DEV_TIMEOUT = 3 };

__device__ __forceinline__ void set_error(int* err, int code, int info) {
  if (atomicCAS(err, 0, code) == 0) err[1] = info;
}

// Storage slot (within one instance) of entry (R_K[p], R_K[q]) for p, q in
// [0, c_K): the diagonal block of J when both rows lie in supernode J, the L
// panel of J = supernode(R_K[q]) when R_K[p] lies in a later supernode, else
// the U^T panel of I = supernode(R_K[p]).  rb = rows_ptr[K].
__device__ __forceinline__ int64_t map_slot(const SymDev& S, int64_t rb, int p, int q) {
  const int bp = S.rows_blk[rb + p];
  const int bq = S.rows_blk[rb + q];
  if (bp >= bq) {
    const int J = S.blk_sn[bq];
    const int64_t base = S.blk_rel[bq] - S.blk_pb[bq];
    const int rp = S.relidx[base + p];
    const int rq = S.relidx[base + q];
    const int sJ = S.sn_width[J];
    if (bp == bq) return S.sn_off[J] + rp + (int64_t)rq * sJ;
    return S.sn_off[J] + (int64_t)sJ * sJ + rp + (int64_t)rq * S.sn_c[J];
  }
  const int I = S.blk_sn[bp];
  const int64_t base = S.blk_rel[bp] - S.blk_pb[bp];
  const int rq = S.relidx[base + q];  // position of R_K[q] in R_I
  const int rp = S.relidx[base + p];  // local column of R_K[p] in I
  const int sI = S.sn_width[I], cI = S.sn_c[I];
  return S.sn_off[I] + (int64_t)sI * sI + (int64_t)cI * sI + rq + (int64_t)rp * cI;
}

// ---------------------------------------------------------------------------
// batched GEMM: C = alpha op(A) op(B) + beta C, or C += alpha op(A) op(B)
// with atomics (split over K).  Column-major operands; op = T reads the
// stored matrix transposed.
// ---------------------------------------------------------------------------
struct GemmDesc {
  const void* A;
  const void* B;
  void* C;
  int M, N, K;
  int lda, ldb, ldc;
  int transA, transB;
  double alpha, beta;
  int atomic;   // 1: atomic accumulation into C (beta ignored)
  int ksplit;   // number of K chunks (tasks carry the chunk index)
  int tri;      // zero structure of the operands: GEMM_TRI_* bits
};
// op(B)(k, n) = 0 for k < n (lower triangular B): a tile needs k >= n0
constexpr int GEMM_TRI_LOWER_B = 1;
// op(A)(m, k) = 0 for k < m (upper triangular A): a tile needs k >= m0
constexpr int GEMM_TRI_UPPER_A = 2;
// op(B)(k, n) = 0 for k > n (upper triangular B): a tile needs k < n0 + BN
constexpr int GEMM_TRI_UPPER_B = 4;
struct GemmTask {
  int d, tm, tn, ks;
};

// per-supernode work item (instance, supernode, extra)
struct SnTask {
  int inst, K, a, b;
};

// contiguous copy segment
struct CopySeg {
  const void* src;
  void* dst;
  int64_t count;  // scalars
};

// ---------------------------------------------------------------------------
// split-precision products (kernels_ozaki.cu)
// ---------------------------------------------------------------------------
enum SliceMode { SLICE_ROWS = 0, SLICE_COLS = 1 };
// One slice set: operand X with R rows (M or N direction) and Kd columns
// (the contracted dimension).  SLICE_ROWS: X(r, k) = src[r + k*ld] (rows of
// the stored column-major matrix); SLICE_COLS: X(r, k) = src[k + r*ld] (its
// columns).  Output: S slices of R64 x K32 tiles of 4 KB, exponents[R].
// Complex sources (cplx = 1): src holds interleaved (re, im) pairs and the
// slice set covers K32 = 2 * ceil(Kd / 32) blocks: the real parts in the
// first half and the imaginary parts in the second, one exponent per row
// for both.
struct SliceDesc {
  const double* src;
  int ld, mode, R, Kd, S, R64, K32, cplx;
  __half* out;
  int* exps;
  unsigned long long* maxbits;  // max_k |X(r,k)| as bit patterns (from the gather or a maxima pass)
};
// one 64-row block and one chunk of 64 K values (two K blocks) of a slice set
struct SliceTask {
  int d, rb, kc;
};
// Complex products use the real embedding: with A = [Re | Im] and
// B = [Re ; Im] slice sets (half = K blocks of one part),
//   Re C: B as stored, MMAs of the second half negated (neg_half = 1),
//   Im C: B halves swapped (swap_b = 1), no negation;
// the result goes to C[(r + n ldc) * cscale + coff] (cscale 2, coff 0 / 1).
struct OzDesc {
  const __half* A;  // slice set of the M x K operand
  const int* eA;
  const __half* B;  // slice set of the N x K operand
  const int* eB;
  double* C;
  int A_R64, B_R64, K32, M, N, ldc, ksplit, atomic;
  int half, swap_b, neg_half, cscale, coff;
  double alpha;
};
struct OzTask {
  int d, tm, tn, ks;
};
// One 64 x 64 tile (tp, tq) of G_K = Ainv(R_K, R_K) of instance `inst`,
// sliced straight from the ancestors' blocks in `store`: dr / dc index the
// SliceDescs of G by rows and by columns (R = Kd = c_K; their src is unused;
// dc < 0: by rows only, for a symmetric G)
struct GTileTask {
  int inst, K, tp, tq, dr, dc;
};
// Running maxima of |Ainv| per global row and column (bit patterns; rowmax
// at rcmax + inst * 2n, colmax n further), the exponents of G's slices:
// every entry of G_K lies in a row and a column whose entries so far
// include it, so the maxima over them bound G's rows and columns.
// maxima = true: the tiles' row and column maxima into rcmax (the G
// blocks a partitioned sweep imports) and the maxima of the ordinary slice
// tasks stasks[0..nst) into their descs' maxbits; false: the tiles' slices
// in both layouts (exponents from rcmax) and the ordinary slices.
void launch_gslice(int dtype, const SymDev& S, const void* store, const SliceDesc* descs,
                   const GTileTask* gtasks, int ngt, const SliceTask* stasks, int nst, bool maxima,
                   unsigned long long* rcmax, cudaStream_t st);
// One chunk of rows of a stored block of Ainv: which = 0 the diagonal
// block of K (rows and columns first(K) + t), 1 a panel whose rows are rows
// of Ainv (entry (p, t) = Ainv(R[p], first + t)), 2 a panel whose rows are
// columns of Ainv (entry (p, t) = Ainv(first + t, R[p])); R from lrows at
// rows_ptr[K] (L panel) or urows at urows_ptr[K] (U^T panel, general).
constexpr int kOutMaxRows = 128;
struct MaxTask {
  int inst, K, which, rc;  // rc: chunk of kOutMaxRows rows
  int64_t off;              // scalar offset of the block in one instance
  int nrows, upanel;        // rows of the block; 1: R from the U^T panel's list
};
// merge the blocks' row and column maxima into rcmax
void launch_out_maxima(int dtype, const SymDev& S, const void* store, const MaxTask* tasks,
                       int ntasks, unsigned long long* rcmax, cudaStream_t st);
cudaError_t prepare_ozaki_kernels();
// maxima = true: accumulate row maxima into desc.maxbits; false: write the slices
void launch_slice(const SliceDesc* descs, const SliceTask* tasks, int ntasks, bool maxima,
                  cudaStream_t st);
// a_tmem: the MMAs read A from tensor memory (copied from the stage per K
// half) instead of shared memory
void launch_ozaki_gemm(int S, const OzDesc* descs, const OzTask* tasks, int ntasks, int* err,
                       bool persistent, bool a_tmem, cudaStream_t st);
void launch_zero(const CopySeg* segs, int nseg, int per_seg, cudaStream_t st);
// a kernel whose only wait never completes: it gives up after budget_ns and
// records DEV_TIMEOUT in err[0]
void launch_wait_selftest(int* err, unsigned long long budget_ns, cudaStream_t st);

// ---------------------------------------------------------------------------
// launch functions (kernels_*.cu)
// ---------------------------------------------------------------------------
enum DType { DT_F64 = 1, DT_C128 = 2 };

// GEMM configurations: tiles (rows x cols of C per CTA) or GEMM_ROWS, row
// panels: one thread per row of C and a chunk of kRowsChunk columns per
// task (64 rows x 8 columns: short tasks, no padding of narrow products,
// and the zero triangle of a triangular op(B) skipped exactly).  Its tasks
// are {d, row block, column chunk, NW + 16 x K chunk}, NW in {4, 8} the
// width the kernel computes for the chunk.
enum GemmCfg { GEMM_64x64 = 0, GEMM_32x32 = 1, GEMM_128x64 = 2, GEMM_ROWS = 3, GEMM_NCFG = 4 };
constexpr int kRowsBlock = 64;
constexpr int kRowsChunk = 8;
// a triangular op(B) (at most one of LOWER_B / UPPER_B) must be square; an
// upper op(A) only goes with a lower op(B)
inline bool rows_eligible(const GemmDesc& d) {
  const int t = d.tri & (GEMM_TRI_LOWER_B | GEMM_TRI_UPPER_B);
  if (t == (GEMM_TRI_LOWER_B | GEMM_TRI_UPPER_B)) return false;
  if (t != 0 && d.N != d.K) return false;
  return !(d.tri & GEMM_TRI_UPPER_A) || t == GEMM_TRI_LOWER_B;
}
void launch_gemm(int dtype, int cfg, const GemmDesc* descs, const GemmTask* tasks, int ntasks,
                 int grid, cudaStream_t st);
int gemm_tile_m(int dtype, int cfg);
int gemm_tile_n(int dtype, int cfg);

// out[p] = sum_b w[b] Ainv_b at entry p of pattern(A) (w: nb device scalars)
void launch_weighted_sum(int dtype, const SymDev& S, const void* store, int nb, const void* w,
                         void* out, cudaStream_t st);
// *out = sum_b w[b] sum_p B[p] Ainv_b at tslot[p] (two launches, fixed reduction
// order; partial: trace_partial_bytes() of device scratch)
void launch_trace(int dtype, const SymDev& S, const void* store, int nb, const void* w,
                  const void* B, const int64_t* tslot, void* partial, void* out, cudaStream_t st);
size_t trace_partial_bytes();
// value scatter (A's entries into the storage of every instance)
void launch_scatter_values(int dtype, const SymDev& S, const void* values, void* store,
                           int nbatch, cudaStream_t st);
// one panel step of the blocked diagonal LU: tasks {inst, K, j0, blk}
// (blk 0: pivot block, 1..nb: rows of L21, nb+1..2nb: columns of U12)
void launch_lu_panel(int dtype, const SymDev& S, void* store, const SnTask* tasks, int ntasks,
                     cudaStream_t st);
// triangular inverses of the diagonal blocks of `store`:
// tasks {inst, K, which (0 = L unit lower, 1 = U upper), first column of a
// panel of 8 columns}; small = 1: blocks of width <= 32, one task per
// triangle (first column 0); result (s x s) at out + wofs[task]
void launch_tri_inv(int dtype, const SymDev& S, const void* store, void* out,
                    const int64_t* wofs, const SnTask* tasks, int ntasks, int max_width,
                    int small, cudaStream_t st);
// FP64 peak loop (the FP64 roofline's denominator): grid for `sms` SMs;
// the launch returns its flops (out: grid * 256 doubles of device scratch)
int fp64_peak_grid(int sms);
double launch_fp64_peak(double* out, int grid, int iters, cudaStream_t st);
// one-time kernel attributes (dynamic shared memory of tri_inv for max_width)
cudaError_t prepare_dense_kernels(int dtype, int max_width);
// G_K = Ainv(R_K, R_K) gathered from `store` into out + gofs[task]
// tasks {inst, K, tile_p, tile_q} (32 x 32 tiles).  With mofs != null
// (real data only), the row and column maxima of |G_K| are also accumulated
// (atomicMax on the bit patterns) into maxbase + mofs[task] (rows, c
// entries) and maxbase + mofs[task] + c (columns).
// Algorithm 1 steps 3-5 of a level of narrow supernodes in one launch, a
// CTA per task {inst, K, j0, w} (c > 0; columns j0 .. j0 + w - 1 of the
// supernode's outputs) with G, Lhat, Uhat^T and w columns of Ainv(C,K) in
// `smem` bytes of shared memory (at most kSmallLevelMaxSmem, see
// small_level_smem); D_K must already be in the diagonal blocks of store
constexpr size_t kSmallLevelMaxSmem = 160 * 1024;
constexpr int kSmallLevelMaxC = 128;
// nblk blocks in R_K, seg relative indices of R_K's blocks
size_t small_level_smem(int dtype, int c, int s, int w, int nblk, int seg);
cudaError_t prepare_map_kernels();
void launch_small_level(int dtype, const SymDev& S, void* store, const void* nf, const SnTask* tasks,
                        int ntasks, size_t smem, int sym, cudaStream_t st);
void launch_gather(int dtype, const SymDev& S, const void* store, void* out,
                   const int64_t* gofs, const SnTask* tasks, int ntasks, cudaStream_t st,
                   const int64_t* mofs = nullptr, unsigned long long* maxbase = nullptr);
// General patterns: G_K = Ainv(R_U(K), R_L(K)) (c_U x c_L, column-major)
// into out + gofs[task], tasks {inst, K, tile over R_U, tile over R_L}
// (32 x 32 tiles); and store(R_L(K), R_U(K)) -= Sc_K (c_L x c_U) from
// src + sofs[task], tasks {inst, K, tile over R_L, tile over R_U}.
void launch_gather_general(int dtype, const SymDev& S, const void* store, void* out,
                           const int64_t* gofs, const SnTask* tasks, int ntasks, cudaStream_t st);
void launch_scatter_sub_general(int dtype, const SymDev& S, void* store, const void* src,
                                const int64_t* sofs, const SnTask* tasks, int ntasks,
                                cudaStream_t st);
// store(R_K, R_K) = src + sofs[task] (the import of a gathered G_K); tasks as for gather
void launch_scatter_set(int dtype, const SymDev& S, void* store, const void* src,
                        const int64_t* sofs, const SnTask* tasks, int ntasks, cudaStream_t st);
// store(R_K, R_K) -= Sc_K (atomic) from src + sofs[task]; tasks as for gather
// lower: only the entries on or below the diagonal of each Sc (p >= q), for
// the symmetric Schur complements of a symmetric A
void launch_scatter_sub(int dtype, const SymDev& S, void* store, const void* src,
                        const int64_t* sofs, const SnTask* tasks, int ntasks, bool lower,
                        cudaStream_t st);
// upper triangle of each task's diagonal block := its lower one, transposed
void launch_mirror_lower(int dtype, const SymDev& S, void* store, const SnTask* tasks, int ntasks,
                         cudaStream_t st);
// per_seg CTAs per segment (the plan sizes it by the longest segment)
void launch_copy(int dtype, const CopySeg* segs, int nseg, int per_seg, cudaStream_t st);
// out[p] = store[inst * storage + value_map[p]]
void launch_extract(int dtype, const SymDev& S, const void* store, int inst, void* out,
                    cudaStream_t st);

}  // namespace pselinv
