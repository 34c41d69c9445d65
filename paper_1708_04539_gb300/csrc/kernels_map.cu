// Index-map kernels (HBM/latency bound): the value scatter into the
// supernodal storage, the gather of Ainv_{C,C} for a supernode (the
// operand of Algorithm 1 steps 3 and 5), the scatter-subtract of a Schur
// complement into the ancestors (supernodal LU), panel copies, and the
// extraction of the selected entries (Algorithm 1 step 6, Theorem 2).
#include "device.cuh"

namespace pselinv {

namespace {

constexpr int kThreads = 256;
constexpr int kTile = 32;

__device__ __forceinline__ bool map_in_range(const SymDev& S, int64_t rb, int p, int q) {
  const int bp = S.rows_blk[rb + p];
  const int bq = S.rows_blk[rb + q];
  const int b = bp >= bq ? bq : bp;
  if (b < 0) return false;
  const int64_t base = S.blk_rel[b] - S.blk_pb[b];
  if (base + p < 0 || base + p >= S.relidx_size || base + q < 0 || base + q >= S.relidx_size)
    return false;
  const int64_t slot = map_slot(S, rb, p, q);
  return slot >= 0 && slot < S.storage;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
scatter_values_kernel(SymDev S, const T* __restrict__ vals, T* store, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / S.nnz, p = e - b * S.nnz;
    store[b * S.storage + S.value_map[p]] = vals[e];
  }
}

__device__ __forceinline__ unsigned long long abs_bits_of(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// One 32 x 32 tile of G_K = Ainv(R_K, R_K) (column-major, ld = c) per task.
// Entries below or on the block diagonal are read down panel columns; the
// ones above it come from U^T panels and are read along their rows, so each
// half of the tile is loaded with the lane index running over the
// contiguous direction and transposed through shared memory.

template <typename T>
__global__ void __launch_bounds__(kThreads)
gather_kernel(SymDev S, const T* __restrict__ store, T* out, const int64_t* __restrict__ gofs,
              const SnTask* __restrict__ tasks, int ntasks, const int64_t* __restrict__ mofs,
              unsigned long long* maxbase) {
  __shared__ T tile[kTile][kTile + 1];
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SnTask task = tasks[t];
    const int K = task.K;
    const int c = S.sn_c[K];
    const int64_t rb = S.rows_ptr[K];
    const T* src = store + (int64_t)task.inst * S.storage;
    T* G = out + gofs[t];
    const int p0 = task.a * kTile, q0 = task.b * kTile;
    // pass 1: lane runs over p (rows): lower/diagonal entries
    for (int r = ly; r < kTile; r += kThreads / 32) {
      const int p = p0 + lx, q = q0 + r;
      if (p < c && q < c && S.rows_blk[rb + p] >= S.rows_blk[rb + q]) {
        if (S.check && !map_in_range(S, rb, p, q)) {
          set_error(S.err, DEV_CHECK, K);
          tile[r][lx] = sc_zero(T());
        } else {
          tile[r][lx] = src[map_slot(S, rb, p, q)];
        }
      }
    }
    // pass 2: lane runs over q (columns): entries from U^T panels
    for (int r = ly; r < kTile; r += kThreads / 32) {
      const int p = p0 + r, q = q0 + lx;
      if (p < c && q < c && S.rows_blk[rb + p] < S.rows_blk[rb + q]) {
        if (S.check && !map_in_range(S, rb, p, q)) {
          set_error(S.err, DEV_CHECK, K);
          tile[lx][r] = sc_zero(T());
        } else {
          tile[lx][r] = src[map_slot(S, rb, p, q)];
        }
      }
    }
    __syncthreads();
    for (int r = ly; r < kTile; r += kThreads / 32) {
      const int p = p0 + lx, q = q0 + r;
      if (p < c && q < c) G[p + (int64_t)q * c] = tile[r][lx];
    }
    if constexpr (sizeof(T) == 8) {
      if (mofs) {
        // row maxima (warp 0: lane = row p) and column maxima (warp 1: lane = column q)
        unsigned long long* mrow = maxbase + mofs[t];
        if (ly == 0 && p0 + lx < c) {
          unsigned long long m = 0;
          for (int q = 0; q < kTile && q0 + q < c; q++) m = max(m, abs_bits_of((double)tile[q][lx]));
          atomicMax(mrow + p0 + lx, m);
        } else if (ly == 1 && q0 + lx < c) {
          unsigned long long m = 0;
          for (int p = 0; p < kTile && p0 + p < c; p++) m = max(m, abs_bits_of((double)tile[lx][p]));
          atomicMax(mrow + c + q0 + lx, m);
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// general patterns (C_L != C_U)
// ---------------------------------------------------------------------------
// Slot of Ainv(x, y) for x = R_U(K)[p] in supernode I (block bp of R_U(K))
// and y = R_L(K)[q] in supernode J (block bq of R_L(K)), on the pattern of
// (L+U)^T: the diagonal block of J (I == J), the U^T panel of J (rows
// R_U(J), I > J) or the L panel of I (rows R_L(I), I < J).  ok = false when
// a checked read falls outside the maps or the storage.
__device__ __forceinline__ int64_t gen_slot(const SymDev& S, int64_t rbL, int64_t rbU, int p,
                                            int q, bool& ok) {
  const int bq = S.rows_blk[rbL + q], bp = S.urows_blk[rbU + p];
  const int J = S.blk_sn[bq], I = S.ublk_sn[bp];
  int64_t ri;
  if (I >= J) {
    ri = S.blk_rel[bq] - S.blk_q0[bq] + p;  // x in J (local) or its position in R_U(J)
  } else {
    ri = S.ublk_rel[bp] - S.ublk_q0[bp] + q;  // position of y in R_L(I)
  }
  if (S.check && (ri < 0 || ri >= S.relidx_size)) {
    ok = false;
    return 0;
  }
  const int64_t r = S.relidx[ri];
  int64_t slot;
  if (I == J) {
    slot = S.sn_off[J] + r + (int64_t)(S.lrows[rbL + q] - S.sn_first[J]) * S.sn_width[J];
  } else if (I > J) {
    const int sJ = S.sn_width[J];
    slot = S.sn_off[J] + (int64_t)sJ * sJ + (int64_t)S.sn_c[J] * sJ + r +
           (int64_t)(S.lrows[rbL + q] - S.sn_first[J]) * S.sn_cu[J];
  } else {
    const int sI = S.sn_width[I];
    slot = S.sn_off[I] + (int64_t)sI * sI + r +
           (int64_t)(S.urows[rbU + p] - S.sn_first[I]) * S.sn_c[I];
  }
  if (S.check && (slot < 0 || slot >= S.storage)) ok = false;
  return slot;
}

// One 32 x 32 tile of G_K = Ainv(R_U(K), R_L(K)) per task: entries with I >= J
// are read down the columns of J's blocks (lanes along p), the others along
// the columns of I's L panel (lanes along q), transposed through shared memory.
template <typename T>
__global__ void __launch_bounds__(kThreads)
gather_general_kernel(SymDev S, const T* __restrict__ store, T* out,
                      const int64_t* __restrict__ gofs, const SnTask* __restrict__ tasks,
                      int ntasks) {
  __shared__ T tile[kTile][kTile + 1];
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SnTask task = tasks[t];
    const int K = task.K;
    const int cl = S.sn_c[K], cu = S.sn_cu[K];
    const int64_t rbL = S.rows_ptr[K], rbU = S.urows_ptr[K];
    const T* src = store + (int64_t)task.inst * S.storage;
    T* G = out + gofs[t];
    const int p0 = task.a * kTile, q0 = task.b * kTile;
    for (int r = ly; r < kTile; r += kThreads / 32) {
      const int p = p0 + lx, q = q0 + r;
      if (p < cu && q < cl &&
          S.ublk_sn[S.urows_blk[rbU + p]] >= S.blk_sn[S.rows_blk[rbL + q]]) {
        bool ok = true;
        const int64_t slot = gen_slot(S, rbL, rbU, p, q, ok);
        if (!ok) set_error(S.err, DEV_CHECK, K);
        tile[r][lx] = ok ? src[slot] : sc_zero(T());
      }
    }
    for (int r = ly; r < kTile; r += kThreads / 32) {
      const int p = p0 + r, q = q0 + lx;
      if (p < cu && q < cl &&
          S.ublk_sn[S.urows_blk[rbU + p]] < S.blk_sn[S.rows_blk[rbL + q]]) {
        bool ok = true;
        const int64_t slot = gen_slot(S, rbL, rbU, p, q, ok);
        if (!ok) set_error(S.err, DEV_CHECK, K);
        tile[lx][r] = ok ? src[slot] : sc_zero(T());
      }
    }
    __syncthreads();
    for (int r = ly; r < kTile; r += kThreads / 32) {
      const int p = p0 + lx, q = q0 + r;
      if (p < cu && q < cl) G[p + (int64_t)q * cu] = tile[r][lx];
    }
    __syncthreads();
  }
}

// store(R_L(K), R_U(K)) -= Sc (c_L x c_U, column-major; atomic: supernodes
// of one level may update the same ancestors).  Entry (i, m), i = R_L[p] in
// supernode I, m = R_U[q] in J, goes to the diagonal block (I == J), the L
// panel of J (I > J: position of i in R_L(J) from the map of R_U(K)'s block)
// or the U^T panel of I (I < J: position of m in R_U(I)).
template <typename T>
__global__ void __launch_bounds__(kThreads)
scatter_sub_general_kernel(SymDev S, T* store, const T* __restrict__ src,
                           const int64_t* __restrict__ sofs, const SnTask* __restrict__ tasks,
                           int ntasks) {
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SnTask task = tasks[t];
    const int K = task.K;
    const int cl = S.sn_c[K], cu = S.sn_cu[K];
    const int64_t rbL = S.rows_ptr[K], rbU = S.urows_ptr[K];
    T* dst = store + (int64_t)task.inst * S.storage;
    const T* Sc = src + sofs[t];
    const int p0 = task.a * kTile, q0 = task.b * kTile;
    for (int r = ly; r < kTile; r += kThreads / 32) {
      const int p = p0 + lx, q = q0 + r;
      if (p >= cl || q >= cu) continue;
      const int bp = S.rows_blk[rbL + p], bq = S.urows_blk[rbU + q];
      const int I = S.blk_sn[bp], J = S.ublk_sn[bq];
      const int i = S.lrows[rbL + p], m = S.urows[rbU + q];
      int64_t slot;
      bool ok = true;
      if (I == J) {
        const int sI = S.sn_width[I], f = S.sn_first[I];
        slot = S.sn_off[I] + (i - f) + (int64_t)(m - f) * sI;
      } else if (I > J) {
        const int64_t ri = S.ublk_rel[bq] - S.ublk_q0[bq] + p;
        if (S.check && (ri < 0 || ri >= S.relidx_size)) ok = false;
        const int sJ = S.sn_width[J];
        slot = ok ? S.sn_off[J] + (int64_t)sJ * sJ + S.relidx[ri] +
                        (int64_t)(m - S.sn_first[J]) * S.sn_c[J]
                  : 0;
      } else {
        const int64_t ri = S.blk_rel[bp] - S.blk_q0[bp] + q;
        if (S.check && (ri < 0 || ri >= S.relidx_size)) ok = false;
        const int sI = S.sn_width[I];
        slot = ok ? S.sn_off[I] + (int64_t)sI * sI + (int64_t)S.sn_c[I] * sI + S.relidx[ri] +
                        (int64_t)(i - S.sn_first[I]) * S.sn_cu[I]
                  : 0;
      }
      if (S.check && (slot < 0 || slot >= S.storage)) ok = false;
      if (!ok) {
        set_error(S.err, DEV_CHECK, K);
        continue;
      }
      atomic_add_s(dst + slot, scale_s(Sc[p + (int64_t)q * cl], -1.0));
    }
  }
}

// store(R_K, R_K) -= Sc (atomic: siblings of one level update shared
// ancestors); ASSIGN: store(R_K, R_K) = Sc (the import of a gathered block);
// LOWER: the entries p >= q only (a symmetric Sc).  Entry (p, q), x = R_K[p]
// in supernode I, y = R_K[q] in J, lies in J's diagonal block or L panel
// (I >= J: the column's storage base + the relative index of p) or in I's
// U^T panel (I < J: the row's base + the relative index of q); the bases of
// the tile's 32 rows and columns are staged in shared memory once, so an
// entry costs one index load, one value load and one store or atomic.
template <typename T, bool ASSIGN = false, bool LOWER = false>
__global__ void __launch_bounds__(kThreads)
scatter_sub_kernel(SymDev S, T* store, const T* __restrict__ src, const int64_t* __restrict__ sofs,
                   const SnTask* __restrict__ tasks, int ntasks) {
  __shared__ int64_t cdiag[kTile], cpan[kTile], crel[kTile], rpan[kTile], rrel[kTile];
  __shared__ int csn[kTile], rsn[kTile];
  const int tid = threadIdx.x, lx = tid & 31, ly = tid >> 5;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SnTask task = tasks[t];
    const int K = task.K;
    const int c = S.sn_c[K];
    const int64_t rb = S.rows_ptr[K];
    T* dst = store + (int64_t)task.inst * S.storage;
    const T* Sc = src + sofs[t];
    const int p0 = task.a * kTile, q0 = task.b * kTile;
    if (tid < kTile) {
      const int q = q0 + tid;
      if (q < c) {
        cdiag[tid] = S.col_diag[rb + q];
        cpan[tid] = S.col_pan[rb + q];
        crel[tid] = S.col_rel[rb + q];
        csn[tid] = S.col_sn[rb + q];
      }
    } else if (tid < 2 * kTile) {
      const int pl = tid - kTile, p = p0 + pl;
      if (p < c) {
        rpan[pl] = S.row_pan[rb + p];
        rrel[pl] = S.row_rel[rb + p];
        rsn[pl] = S.row_sn[rb + p];
      }
    }
    __syncthreads();
    for (int r = ly; r < kTile; r += kThreads / 32) {
      const int p = p0 + lx, q = q0 + r;  // lanes along p: Sc is column major
      if (p >= c || q >= c || (LOWER && p < q)) continue;
      const bool col_side = rsn[lx] >= csn[r];
      const int64_t ri = col_side ? crel[r] + p : rrel[lx] + q;
      if (S.check && (ri < 0 || ri >= S.relidx_size)) {
        set_error(S.err, DEV_CHECK, K);
        continue;
      }
      const int64_t slot =
          (col_side ? (rsn[lx] == csn[r] ? cdiag[r] : cpan[r]) : rpan[lx]) + S.relidx[ri];
      if (S.check && (slot < 0 || slot >= S.storage)) {
        set_error(S.err, DEV_CHECK, K);
        continue;
      }
      const T v = Sc[p + (int64_t)q * c];
      if (ASSIGN)
        dst[slot] = v;
      else
        atomic_add_s(dst + slot, scale_s(v, -1.0));
    }
    __syncthreads();
  }
}

// D(i, j) = D(j, i) for i < j of the diagonal block of each task's
// supernode: 32 x 32 tiles of the upper triangle staged through shared
// memory (coalesced on both sides)
template <typename T>
__global__ void __launch_bounds__(kThreads)
mirror_lower_kernel(SymDev S, T* store, const SnTask* __restrict__ tasks, int ntasks) {
  __shared__ T tile[kTile][kTile + 1];
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SnTask task = tasks[t];
    const int s = S.sn_width[task.K];
    T* D = store + (int64_t)task.inst * S.storage + S.sn_off[task.K];
    const int nb = (s + kTile - 1) / kTile;
    for (int bj = 0; bj < nb; bj++)
      for (int bi = 0; bi <= bj; bi++) {
        // source: rows bj*32.., columns bi*32.. (on or below the diagonal)
        for (int r = ly; r < kTile; r += kThreads / 32) {
          const int row = bj * kTile + lx, col = bi * kTile + r;
          if (row < s && col < s) tile[r][lx] = D[row + (int64_t)col * s];
        }
        __syncthreads();
        // destination: rows bi*32.., columns bj*32.., entries above the diagonal
        for (int r = ly; r < kTile; r += kThreads / 32) {
          const int row = bi * kTile + lx, col = bj * kTile + r;
          if (row < s && col < s && row < col) D[row + (int64_t)col * s] = tile[lx][r];
        }
        __syncthreads();
      }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
copy_kernel(const CopySeg* __restrict__ segs, int nseg) {
  for (int s = blockIdx.y; s < nseg; s += gridDim.y) {
    const CopySeg g = segs[s];
    const T* a = (const T*)g.src;
    T* b = (T*)g.dst;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.count;
         e += (int64_t)gridDim.x * blockDim.x)
      b[e] = a[e];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
extract_kernel(SymDev S, const T* __restrict__ store, T* out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < S.nnz;
       p += (int64_t)gridDim.x * blockDim.x)
    out[p] = store[S.out_map[p]];
}

// Pole-expansion consumers (a weighted sum over the instances of a batch).
// out[p] = sum_b w_b Ainv_b at entry p of pattern(A).
template <typename T>
__global__ void __launch_bounds__(kThreads)
weighted_sum_kernel(SymDev S, const T* __restrict__ store, int nb, const T* __restrict__ w,
                    T* out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < S.nnz;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t slot = S.out_map[p];
    T acc = sc_zero(T());
    for (int b = 0; b < nb; b++) acc = add_s(acc, mul_s(w[b], store[b * S.storage + slot]));
    out[p] = acc;
  }
}

// Partial sums of sum_b w_b sum_p B[p] Ainv_b(j, i) for entry p = (i, j) of
// pattern(A) (tslot[p] = storage slot of the transposed entry): a fixed grid
// and a fixed reduction order, so the result does not depend on timing.
constexpr int kTraceBlocks = 1024;
template <typename T>
__global__ void __launch_bounds__(kThreads)
trace_partial_kernel(SymDev S, const T* __restrict__ store, int nb, const T* __restrict__ w,
                     const T* __restrict__ B, const int64_t* __restrict__ tslot, T* partial) {
  __shared__ T red[kThreads];
  T acc = sc_zero(T());
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < S.nnz;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t slot = tslot[p];
    T x = sc_zero(T());
    for (int b = 0; b < nb; b++) x = add_s(x, mul_s(w[b], store[b * S.storage + slot]));
    acc = add_s(acc, mul_s(B[p], x));
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = add_s(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

template <typename T>
__global__ void __launch_bounds__(kThreads) trace_final_kernel(const T* __restrict__ partial, T* out) {
  __shared__ T red[kThreads];
  T acc = sc_zero(T());
  for (int i = threadIdx.x; i < kTraceBlocks; i += kThreads) acc = add_s(acc, partial[i]);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = add_s(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Algorithm 1 steps 3-5 of an FP64 level of narrow supernodes in one
// launch.  A task {inst, K, j0, w} owns columns j0 .. j0 + w - 1 of the
// supernode's outputs: G = Ainv(R_K, R_K) is gathered into shared memory
// (leading dimension ldg = c | 1, so that the transposed reads of step 5
// spread over the banks) with Lhat and Uhat^T (c x s); then Ainv(C,K) = -G
// Lhat and Ainv(K,C)^T = -G^T Uhat^T for those columns into the panels (for
// a symmetric A the second is a copy of the first) and Ainv_KK(:, j) = D_K(:,
// j) - Uhat Ainv(C,K)(:, j) onto the diagonal block (D_K written there by
// the normalisation).  Dot products over c from shared memory; the tasks
// of a supernode write disjoint columns, so no atomics.
template <typename T>
__global__ void __launch_bounds__(kThreads)
small_level_kernel(SymDev S, T* store, const T* __restrict__ nf, const SnTask* __restrict__ tasks,
                   int ntasks, int sym) {
  extern __shared__ __align__(16) unsigned char small_smem[];
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SnTask task = tasks[t];
    const int K = task.K, j0 = task.a, w = task.b;
    const int c = S.sn_c[K], s = S.sn_width[K];
    const int ldg = c | 1;
    const int64_t rb = S.rows_ptr[K];
    const int64_t base = (int64_t)task.inst * S.storage;
    const int64_t so = base + S.sn_off[K], lo = so + (int64_t)s * s, uo = lo + (int64_t)c * s;
    // index tables of R_K's blocks (consecutive block ids b0 ..): the local
    // block of every position, the supernode's relative-index segment, and
    // per block the storage offset, width and |R| of its supernode and the
    // start of its relative indices within the segment
    const int b0 = S.rows_blk[rb], nblk = S.rows_blk[rb + c - 1] - b0 + 1;
    const int64_t rel0 = S.blk_rel[b0];
    const int seg = (int)(S.blk_rel[b0 + nblk - 1] + (c - S.blk_pb[b0 + nblk - 1]) - rel0);
    int64_t* m_off = reinterpret_cast<int64_t*>(small_smem);
    int* m_s = reinterpret_cast<int*>(m_off + nblk);
    int* m_c = m_s + nblk;
    int* m_base = m_c + nblk;
    int* lblk = m_base + nblk;
    int* rel = lblk + c;
    const size_t ibytes = ((size_t)nblk * 20 + (size_t)(c + seg) * 4 + 15) & ~size_t(15);
    T* G = reinterpret_cast<T*>(small_smem + ibytes);
    T* Lh = G + (int64_t)ldg * c;
    T* Uh = Lh + (int64_t)c * s;
    T* X = Uh + (int64_t)c * s;  // c x w: Ainv(C,K)(:, j0 .. j0 + w - 1)
    for (int l = threadIdx.x; l < nblk; l += blockDim.x) {
      const int J = S.blk_sn[b0 + l];
      m_off[l] = S.sn_off[J];
      m_s[l] = S.sn_width[J];
      m_c[l] = S.sn_c[J];
      m_base[l] = (int)(S.blk_rel[b0 + l] - rel0) - S.blk_pb[b0 + l];
    }
    for (int p = threadIdx.x; p < c; p += blockDim.x) lblk[p] = S.rows_blk[rb + p] - b0;
    for (int i = threadIdx.x; i < seg; i += blockDim.x) rel[i] = S.relidx[rel0 + i];
    for (int e = threadIdx.x; e < c * s; e += blockDim.x) {
      Lh[e] = nf[lo + e];
      if (!sym) Uh[e] = nf[uo + e];
    }
    __syncthreads();
    // G = Ainv(R_K, R_K): the slot of (p, q) as in map_slot, from the tables
    const T* src = store + base;
    for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
      const int p = e % c, q = e / c;
      T v = sc_zero(T());
      if (S.check) {
        if (!map_in_range(S, rb, p, q))
          set_error(S.err, DEV_CHECK, K);
        else
          v = src[map_slot(S, rb, p, q)];
      } else {
        const int lp = lblk[p], lq = lblk[q], l = lp < lq ? lp : lq;
        const int rp = rel[m_base[l] + p], rq = rel[m_base[l] + q];
        const int64_t sJ = m_s[l], cJ = m_c[l];
        int64_t slot;
        if (lp == lq)
          slot = m_off[l] + rp + rq * sJ;
        else if (lp > lq)
          slot = m_off[l] + sJ * sJ + rp + rq * cJ;
        else
          slot = m_off[l] + sJ * sJ + cJ * sJ + rq + rp * cJ;
        v = src[slot];
      }
      G[p + q * ldg] = v;
    }
    __syncthreads();
    // steps 3 and 5
    for (int e = threadIdx.x; e < c * w; e += blockDim.x) {
      const int p = e % c, j = j0 + e / c;
      T a = sc_zero(T()), b = sc_zero(T());
      for (int q = 0; q < c; q++) {
        a = fma_s(G[p + q * ldg], Lh[q + j * c], a);
        if (!sym) b = fma_s(G[q + p * ldg], Uh[q + j * c], b);
      }
      a = scale_s(a, -1.0);
      X[e] = a;
      store[lo + p + (int64_t)j * c] = a;
      store[uo + p + (int64_t)j * c] = sym ? a : scale_s(b, -1.0);
    }
    __syncthreads();
    // step 4 (symmetric A: Uhat^T = Lhat)
    const T* A4 = sym ? Lh : Uh;
    for (int e = threadIdx.x; e < s * w; e += blockDim.x) {
      const int i = e % s, jj = e / s;
      T a = sc_zero(T());
      for (int q = 0; q < c; q++) a = fma_s(A4[q + i * c], X[q + jj * c], a);
      T* d = store + so + i + (int64_t)(j0 + jj) * s;
      *d = sub_s(*d, a);
    }
    __syncthreads();
  }
}

int grid_for(int64_t n) {
  const int64_t g = (n + kThreads - 1) / kThreads;
  return (int)(g < 152 * 16 ? (g > 0 ? g : 1) : 152 * 16);
}

}  // namespace

void launch_scatter_values(int dtype, const SymDev& S, const void* values, void* store,
                           int nbatch, cudaStream_t st) {
  const int64_t total = (int64_t)nbatch * S.nnz;
  if (total == 0) return;
  if (dtype == DT_F64)
    scatter_values_kernel<double><<<grid_for(total), kThreads, 0, st>>>(S, (const double*)values,
                                                                      (double*)store, total);
  else
    scatter_values_kernel<cdouble><<<grid_for(total), kThreads, 0, st>>>(
        S, (const cdouble*)values, (cdouble*)store, total);
}

size_t small_level_smem(int dtype, int c, int s, int w, int nblk, int seg) {
  const size_t ibytes = ((size_t)nblk * 20 + (size_t)(c + seg) * 4 + 15) & ~size_t(15);
  return ibytes + (size_t)((int64_t)(c | 1) * c + 2 * (int64_t)c * s + (int64_t)c * w) *
                      (dtype == DT_F64 ? 8 : 16);
}

cudaError_t prepare_map_kernels() {
  cudaError_t e = cudaFuncSetAttribute(small_level_kernel<double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSmallLevelMaxSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(small_level_kernel<cdouble>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallLevelMaxSmem);
}

void launch_small_level(int dtype, const SymDev& S, void* store, const void* nf, const SnTask* tasks,
                        int ntasks, size_t smem, int sym, cudaStream_t st) {
  if (ntasks <= 0) return;
  if (dtype == DT_F64)
    small_level_kernel<double><<<ntasks, kThreads, smem, st>>>(S, (double*)store, (const double*)nf,
                                                               tasks, ntasks, sym);
  else
    small_level_kernel<cdouble><<<ntasks, kThreads, smem, st>>>(S, (cdouble*)store,
                                                                (const cdouble*)nf, tasks, ntasks, sym);
}

void launch_gather(int dtype, const SymDev& S, const void* store, void* out, const int64_t* gofs,
                   const SnTask* tasks, int ntasks, cudaStream_t st, const int64_t* mofs,
                   unsigned long long* maxbase) {
  if (ntasks <= 0) return;
  const int grid = ntasks < 152 * 8 ? ntasks : 152 * 8;
  if (dtype == DT_F64)
    gather_kernel<double><<<grid, kThreads, 0, st>>>(S, (const double*)store, (double*)out, gofs,
                                                     tasks, ntasks, mofs, maxbase);
  else
    gather_kernel<cdouble><<<grid, kThreads, 0, st>>>(S, (const cdouble*)store, (cdouble*)out,
                                                      gofs, tasks, ntasks, nullptr, nullptr);
}

void launch_scatter_sub(int dtype, const SymDev& S, void* store, const void* src,
                        const int64_t* sofs, const SnTask* tasks, int ntasks, bool lower,
                        cudaStream_t st) {
  if (ntasks <= 0) return;
  const int grid = ntasks < 152 * 8 ? ntasks : 152 * 8;
  if (dtype == DT_F64) {
    if (lower)
      scatter_sub_kernel<double, false, true><<<grid, kThreads, 0, st>>>(
          S, (double*)store, (const double*)src, sofs, tasks, ntasks);
    else
      scatter_sub_kernel<double><<<grid, kThreads, 0, st>>>(S, (double*)store,
                                                            (const double*)src, sofs, tasks, ntasks);
  } else {
    if (lower)
      scatter_sub_kernel<cdouble, false, true><<<grid, kThreads, 0, st>>>(
          S, (cdouble*)store, (const cdouble*)src, sofs, tasks, ntasks);
    else
      scatter_sub_kernel<cdouble><<<grid, kThreads, 0, st>>>(
          S, (cdouble*)store, (const cdouble*)src, sofs, tasks, ntasks);
  }
}

void launch_mirror_lower(int dtype, const SymDev& S, void* store, const SnTask* tasks, int ntasks,
                         cudaStream_t st) {
  if (ntasks <= 0) return;
  const int grid = ntasks < 152 * 8 ? ntasks : 152 * 8;
  if (dtype == DT_F64)
    mirror_lower_kernel<double><<<grid, kThreads, 0, st>>>(S, (double*)store, tasks, ntasks);
  else
    mirror_lower_kernel<cdouble><<<grid, kThreads, 0, st>>>(S, (cdouble*)store, tasks, ntasks);
}

void launch_gather_general(int dtype, const SymDev& S, const void* store, void* out,
                           const int64_t* gofs, const SnTask* tasks, int ntasks, cudaStream_t st) {
  if (ntasks <= 0) return;
  const int grid = ntasks < 152 * 8 ? ntasks : 152 * 8;
  if (dtype == DT_F64)
    gather_general_kernel<double><<<grid, kThreads, 0, st>>>(S, (const double*)store,
                                                             (double*)out, gofs, tasks, ntasks);
  else
    gather_general_kernel<cdouble><<<grid, kThreads, 0, st>>>(S, (const cdouble*)store,
                                                              (cdouble*)out, gofs, tasks, ntasks);
}

void launch_scatter_sub_general(int dtype, const SymDev& S, void* store, const void* src,
                                const int64_t* sofs, const SnTask* tasks, int ntasks,
                                cudaStream_t st) {
  if (ntasks <= 0) return;
  const int grid = ntasks < 152 * 8 ? ntasks : 152 * 8;
  if (dtype == DT_F64)
    scatter_sub_general_kernel<double><<<grid, kThreads, 0, st>>>(
        S, (double*)store, (const double*)src, sofs, tasks, ntasks);
  else
    scatter_sub_general_kernel<cdouble><<<grid, kThreads, 0, st>>>(
        S, (cdouble*)store, (const cdouble*)src, sofs, tasks, ntasks);
}

void launch_scatter_set(int dtype, const SymDev& S, void* store, const void* src,
                        const int64_t* sofs, const SnTask* tasks, int ntasks, cudaStream_t st) {
  if (ntasks <= 0) return;
  const int grid = ntasks < 152 * 8 ? ntasks : 152 * 8;
  if (dtype == DT_F64)
    scatter_sub_kernel<double, true><<<grid, kThreads, 0, st>>>(
        S, (double*)store, (const double*)src, sofs, tasks, ntasks);
  else
    scatter_sub_kernel<cdouble, true><<<grid, kThreads, 0, st>>>(
        S, (cdouble*)store, (const cdouble*)src, sofs, tasks, ntasks);
}

void launch_copy(int dtype, const CopySeg* segs, int nseg, int per_seg, cudaStream_t st) {
  if (nseg <= 0) return;
  dim3 grid(per_seg > 0 ? per_seg : 8, nseg < 65535 ? nseg : 65535);
  if (dtype == DT_F64)
    copy_kernel<double><<<grid, kThreads, 0, st>>>(segs, nseg);
  else
    copy_kernel<cdouble><<<grid, kThreads, 0, st>>>(segs, nseg);
}

void launch_extract(int dtype, const SymDev& S, const void* store, int inst, void* out,
                    cudaStream_t st) {
  if (S.nnz == 0) return;
  if (dtype == DT_F64)
    extract_kernel<double><<<grid_for(S.nnz), kThreads, 0, st>>>(
        S, (const double*)store + (int64_t)inst * S.storage, (double*)out);
  else
    extract_kernel<cdouble><<<grid_for(S.nnz), kThreads, 0, st>>>(
        S, (const cdouble*)store + (int64_t)inst * S.storage, (cdouble*)out);
}

void launch_weighted_sum(int dtype, const SymDev& S, const void* store, int nb, const void* w,
                         void* out, cudaStream_t st) {
  if (S.nnz == 0) return;
  if (dtype == DT_F64)
    weighted_sum_kernel<double><<<grid_for(S.nnz), kThreads, 0, st>>>(
        S, (const double*)store, nb, (const double*)w, (double*)out);
  else
    weighted_sum_kernel<cdouble><<<grid_for(S.nnz), kThreads, 0, st>>>(
        S, (const cdouble*)store, nb, (const cdouble*)w, (cdouble*)out);
}

void launch_trace(int dtype, const SymDev& S, const void* store, int nb, const void* w,
                  const void* B, const int64_t* tslot, void* partial, void* out, cudaStream_t st) {
  if (dtype == DT_F64) {
    trace_partial_kernel<double><<<kTraceBlocks, kThreads, 0, st>>>(
        S, (const double*)store, nb, (const double*)w, (const double*)B, tslot, (double*)partial);
    trace_final_kernel<double><<<1, kThreads, 0, st>>>((const double*)partial, (double*)out);
  } else {
    trace_partial_kernel<cdouble><<<kTraceBlocks, kThreads, 0, st>>>(
        S, (const cdouble*)store, nb, (const cdouble*)w, (const cdouble*)B, tslot,
        (cdouble*)partial);
    trace_final_kernel<cdouble><<<1, kThreads, 0, st>>>((const cdouble*)partial, (cdouble*)out);
  }
}

size_t trace_partial_bytes() { return (size_t)kTraceBlocks * 16; }

}  // namespace pselinv
