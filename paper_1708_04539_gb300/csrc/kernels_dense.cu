// Dense block kernels in FP64 / complex128:
//   * a batched, persistent GEMM over a task list (the block products of
//     Algorithm 1 steps 2-5 and of the supernodal LU),
//   * the panel steps of the blocked LU without pivoting of diagonal blocks,
//   * triangular inverses of the diagonal blocks (one warp per column).
//
// On GB300 the FP64 rate is the same for DFMA and the FP64 MMA path (about
// 4 flop/clk/SM), so the FP64 GEMM is a register-tiled SIMT DFMA kernel:
// it saturates the FP64 pipe with a 16x16 thread grid and 4x4 (real) or
// 2x2 (complex) outputs per thread.
#include "device.cuh"

namespace pselinv {

namespace {

constexpr int kThreads = 256;

template <typename T, int BM, int BN, int BK>
struct GemmSmem {
  T a[BK][BM];
  T b[BK][BN];
};

template <typename T, int BM, int BN, int BK>
__global__ void __launch_bounds__(kThreads)
gemm_kernel(const GemmDesc* __restrict__ descs, const GemmTask* __restrict__ tasks, int ntasks) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ GemmSmem<T, BM, BN, BK> sm;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const GemmTask task = tasks[t];
    const GemmDesc d = descs[task.d];
    const T* __restrict__ A = (const T*)d.A;
    const T* __restrict__ B = (const T*)d.B;
    T* __restrict__ C = (T*)d.C;
    const int m0 = task.tm * BM, n0 = task.tn * BN;
    int kchunk = (d.K + d.ksplit - 1) / d.ksplit;
    kchunk = (kchunk + BK - 1) / BK * BK;
    int kb = task.ks * kchunk;
    int ke = min(d.K, kb + kchunk);
    if (d.tri & GEMM_TRI_LOWER_B) kb = max(kb, n0);
    if (d.tri & GEMM_TRI_UPPER_A) kb = max(kb, m0);
    if (d.tri & GEMM_TRI_UPPER_B) ke = min(ke, n0 + BN);
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
      for (int j = 0; j < TN; j++) acc[i][j] = sc_zero(T());
    // the next K tile is loaded into registers while the current one is
    // used from shared memory
    constexpr int NA = BM * BK / kThreads, NB = BK * BN / kThreads;
    T ra[NA], rb[NB];
    auto load_tiles = [&](int k0) {
#pragma unroll
      for (int q = 0; q < NA; q++) {
        const int e = tid + q * kThreads;
        int mm, kk;
        if (d.transA) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
        const int m = m0 + mm, k = k0 + kk;
        T v = sc_zero(T());
        if (m < d.M && k < ke)
          v = d.transA ? A[k + (int64_t)m * d.lda] : A[m + (int64_t)k * d.lda];
        ra[q] = v;
      }
#pragma unroll
      for (int q = 0; q < NB; q++) {
        const int e = tid + q * kThreads;
        int kk, nn;
        if (d.transB) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
        const int n = n0 + nn, k = k0 + kk;
        T v = sc_zero(T());
        if (n < d.N && k < ke)
          v = d.transB ? B[n + (int64_t)k * d.ldb] : B[k + (int64_t)n * d.ldb];
        rb[q] = v;
      }
    };
    if (kb < ke) load_tiles(kb);
    for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
      for (int q = 0; q < NA; q++) {
        const int e = tid + q * kThreads;
        if (d.transA) sm.a[e % BK][e / BK] = ra[q]; else sm.a[e / BM][e % BM] = ra[q];
      }
#pragma unroll
      for (int q = 0; q < NB; q++) {
        const int e = tid + q * kThreads;
        if (d.transB) sm.b[e / BN][e % BN] = rb[q]; else sm.b[e % BK][e / BK] = rb[q];
      }
      __syncthreads();
      if (k0 + BK < ke) load_tiles(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; kk++) {
        T av[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; i++) av[i] = sm.a[kk][tx + 16 * i];
#pragma unroll
        for (int j = 0; j < TN; j++) bv[j] = sm.b[kk][ty + 16 * j];
#pragma unroll
        for (int i = 0; i < TM; i++)
#pragma unroll
          for (int j = 0; j < TN; j++) acc[i][j] = fma_s(av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; i++) {
      const int m = m0 + tx + 16 * i;
      if (m >= d.M) continue;
#pragma unroll
      for (int j = 0; j < TN; j++) {
        const int n = n0 + ty + 16 * j;
        if (n >= d.N) continue;
        T* c = C + m + (int64_t)n * d.ldc;
        const T v = scale_s(acc[i][j], d.alpha);
        if (d.atomic) {
          atomic_add_s(c, v);
        } else if (d.beta != 0.0) {
          *c = add_s(v, scale_s(*c, d.beta));
        } else {
          *c = v;
        }
      }
    }
  }
}

// Panel step of the blocked LU without pivoting of the s x s diagonal
// block of a supernode (right-looking, panels of 32 columns; the trailing
// update A22 -= L21 U12 is a GEMM launch of its own).  Task {inst, K, j0,
// blk} with w = min(32, s - j0) and nb = number of 32-blocks below the
// pivot block: blk = 0 factors the w x w pivot block at (j0, j0) in shared
// memory and writes it back (a launch of its own, before the others read
// it); blk in [1, nb] solves the 32 rows j0 + w + 32 (blk - 1) .. of
// L21 = A21 U11^{-1}, blk in [nb + 1, 2 nb] the 32 columns of
// U12 = L11^{-1} A12.  One division per pivot and CTA.
template <typename T>
__global__ void __launch_bounds__(kThreads)
lu_panel_kernel(SymDev S, T* store, const SnTask* __restrict__ tasks, int ntasks) {
  __shared__ T Dd[32][33];
  __shared__ T R[32];
  __shared__ T X[32][33];
  const int tid = threadIdx.x;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SnTask task = tasks[t];
    const int K = task.K;
    const int s = S.sn_width[K];
    const int j0 = task.a, blk = task.b;
    const int w = min(32, s - j0);
    T* D = store + (int64_t)task.inst * S.storage + S.sn_off[K];
    for (int e = tid; e < w * w; e += kThreads) {
      const int i = e % w, j = e / w;
      Dd[i][j] = D[(j0 + i) + (int64_t)(j0 + j) * s];
    }
    __syncthreads();
    const int nb = (s - j0 - w + 31) / 32;
    if (blk == 0) {
      for (int k = 0; k < w; k++) {
        if (tid == 0) {
          const T piv = Dd[k][k];
          if (is_zero(piv)) set_error(S.err, DEV_ZERO_PIVOT, S.sn_first[K] + j0 + k);
          R[k] = div_s(sc_one(T()), piv);
        }
        __syncthreads();
        for (int i = k + 1 + tid; i < w; i += kThreads) Dd[i][k] = mul_s(Dd[i][k], R[k]);
        __syncthreads();
        const int m = w - k - 1;
        for (int e = tid; e < m * m; e += kThreads) {
          const int i = k + 1 + e % m, j = k + 1 + e / m;
          Dd[i][j] = sub_s(Dd[i][j], mul_s(Dd[i][k], Dd[k][j]));
        }
        __syncthreads();
      }
      for (int e = tid; e < w * w; e += kThreads) {
        const int i = e % w, j = e / w;
        D[(j0 + i) + (int64_t)(j0 + j) * s] = Dd[i][j];
      }
      __syncthreads();
      continue;
    }
    // the pivot block is factored already: L11 below, U11 on and above
    if (tid < w) R[tid] = div_s(sc_one(T()), Dd[tid][tid]);
    __syncthreads();
    if (blk <= nb) {
      // rows of L21: X U11 = A21, one column of X at a time
      const int r0 = j0 + w + 32 * (blk - 1), nr = min(32, s - r0);
      for (int e = tid; e < nr * w; e += kThreads) {
        const int i = e % nr, j = e / nr;
        X[i][j] = D[(r0 + i) + (int64_t)(j0 + j) * s];
      }
      __syncthreads();
      for (int j = 0; j < w; j++) {
        for (int i = tid; i < nr; i += kThreads) X[i][j] = mul_s(X[i][j], R[j]);
        __syncthreads();
        const int m = w - j - 1;
        for (int e = tid; e < nr * m; e += kThreads) {
          const int i = e % nr, kk = j + 1 + e / nr;
          X[i][kk] = sub_s(X[i][kk], mul_s(X[i][j], Dd[j][kk]));
        }
        __syncthreads();
      }
      for (int e = tid; e < nr * w; e += kThreads) {
        const int i = e % nr, j = e / nr;
        D[(r0 + i) + (int64_t)(j0 + j) * s] = X[i][j];
      }
    } else {
      // columns of U12: L11 Y = A12 (unit lower), one row of Y at a time
      const int c0 = j0 + w + 32 * (blk - nb - 1), nc = min(32, s - c0);
      for (int e = tid; e < w * nc; e += kThreads) {
        const int i = e % w, j = e / w;
        X[i][j] = D[(j0 + i) + (int64_t)(c0 + j) * s];
      }
      __syncthreads();
      for (int k = 0; k < w - 1; k++) {
        const int m = w - k - 1;
        for (int e = tid; e < m * nc; e += kThreads) {
          const int i = k + 1 + e % m, j = e / m;
          X[i][j] = sub_s(X[i][j], mul_s(Dd[i][k], X[k][j]));
        }
        __syncthreads();
      }
      for (int e = tid; e < w * nc; e += kThreads) {
        const int i = e % w, j = e / w;
        D[(j0 + i) + (int64_t)(c0 + j) * s] = X[i][j];
      }
    }
    __syncthreads();
  }
}

// Triangular inverses of the diagonal blocks: which = 0 gives (L_KK)^{-1}
// (unit lower), which = 1 gives (U_KK)^{-1} (upper), column j of the
// inverse being the solution of a triangular system with right-hand side
// e_j.  FP64 runs at about 4 flop/clk/SM on this GPU, so a launch is fast
// only when its solves are spread over many SMs and the FP64 pipe is all a
// solve waits on: one warp per column, the column in registers (lane l holds
// rows l, l + 32, ...), the factor streamed through shared memory for the
// eight columns (warps) of a CTA, and no block barrier inside a chunk.
constexpr int kTriChunk = 8;   // factor columns staged per shared-memory pass
constexpr int kTriRb = 8;      // 32-row blocks per column (s <= 256)
constexpr int kTriSmallS = 32; // blocks this wide or narrower: one warp per triangle

__device__ __forceinline__ double shfl_s(double v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
__device__ __forceinline__ cdouble shfl_s(cdouble v, int src) {
  return {__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}

// s > 32: a task is a panel of 8 consecutive columns j0.. (warp w solves
// column j0 + w); the factor goes through shared memory kTriChunk columns at
// a time.
template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
tri_inv_kernel(SymDev S, const T* store, T* out, const int64_t* __restrict__ wofs,
               const SnTask* __restrict__ tasks, int ntasks) {
  __shared__ T F[kTriChunk][kTriRb * 32];
  __shared__ T R[kTriChunk];  // reciprocals of the chunk's diagonal entries of U
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SnTask task = tasks[t];
    const int K = task.K;
    const int s = S.sn_width[K];
    const int nrb = (s + 31) >> 5;
    const int j0 = task.b;
    const int col = j0 + w;  // >= s: idle warp (still takes part in the barriers)
    const T* D = store + (int64_t)task.inst * S.storage + S.sn_off[K];
    T x[kTriRb];
#pragma unroll
    for (int m = 0; m < kTriRb; m++) x[m] = (lane + 32 * m == col) ? sc_one(T()) : sc_zero(T());
    if (task.a == 0) {
      // L x = e_col, forward: rows below k take x_k once it is final
      for (int k0 = j0; k0 < s - 1; k0 += kTriChunk) {
        const int kn = min(kTriChunk, s - 1 - k0);
        __syncthreads();
        for (int e = threadIdx.x; e < kn * s; e += kThreads) {
          const int kk = e / s, i = e - kk * s;
          F[kk][i] = D[i + (int64_t)(k0 + kk) * s];
        }
        __syncthreads();
        for (int kk = 0; kk < kn; kk++) {
          const int k = k0 + kk, mk = k >> 5;
          T v = x[0];
#pragma unroll
          for (int m = 1; m < kTriRb; m++)
            if (m == mk) v = x[m];
          const T xk = shfl_s(v, k & 31);
#pragma unroll
          for (int m = 0; m < kTriRb; m++) {
            if (m >= mk && m < nrb) {
              const int i = lane + 32 * m;
              if (i > k && i < s) x[m] = sub_s(x[m], mul_s(F[kk][i], xk));
            }
          }
        }
      }
    } else {
      // U x = e_col, backward from the panel's last column
      const int kend = min(j0 + kThreads / 32, s) - 1;
      for (int k0 = kend; k0 >= 0; k0 -= kTriChunk) {
        const int kn = min(kTriChunk, k0 + 1);
        __syncthreads();
        for (int e = threadIdx.x; e < kn * (k0 + 1); e += kThreads) {
          const int kk = e / (k0 + 1), i = e - kk * (k0 + 1);
          F[kk][i] = D[i + (int64_t)(k0 - kk) * s];
        }
        // one division per diagonal entry and CTA: an FP64 division is a
        // sequence of FP64 operations, too dear to repeat in every column
        if (threadIdx.x < kn) {
          const T u = D[(k0 - threadIdx.x) + (int64_t)(k0 - threadIdx.x) * s];
          if (is_zero(u)) set_error(S.err, DEV_ZERO_PIVOT, S.sn_first[K] + k0 - threadIdx.x);
          R[threadIdx.x] = div_s(sc_one(T()), u);
        }
        __syncthreads();
        for (int kk = 0; kk < kn; kk++) {
          const int k = k0 - kk, mk = k >> 5;
          T v = x[0];
#pragma unroll
          for (int m = 1; m < kTriRb; m++)
            if (m == mk) v = x[m];
          const T xk = mul_s(shfl_s(v, k & 31), R[kk]);
#pragma unroll
          for (int m = 0; m < kTriRb; m++) {
            if (m <= mk) {
              const int i = lane + 32 * m;
              if (i == k) x[m] = xk;
              else if (i < k) x[m] = sub_s(x[m], mul_s(F[kk][i], xk));
            }
          }
        }
      }
    }
    if (col < s) {
      T* W = out + wofs[t] + (int64_t)col * s;
#pragma unroll
      for (int m = 0; m < kTriRb; m++) {
        const int i = lane + 32 * m;
        if (m < nrb && i < s) W[i] = x[m];
      }
    }
  }
}

// s <= 32: one warp inverts one triangle, lane j solving column j with the
// column in registers; every lane reads the same factor entry (a broadcast
// load), and the unrolled loops let those loads run ahead of the solve.
template <typename T>
__global__ void __launch_bounds__(kThreads)
tri_inv_small_kernel(SymDev S, const T* store, T* out, const int64_t* __restrict__ wofs,
                     const SnTask* __restrict__ tasks, int ntasks) {
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (kThreads / 32);
  for (int t = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); t < ntasks; t += nwarps) {
    const SnTask task = tasks[t];
    const int K = task.K;
    const int s = S.sn_width[K];
    const T* __restrict__ D = store + (int64_t)task.inst * S.storage + S.sn_off[K];
    T x[kTriSmallS];
#pragma unroll
    for (int i = 0; i < kTriSmallS; i++) x[i] = (i == lane) ? sc_one(T()) : sc_zero(T());
    if (task.a == 0) {
#pragma unroll
      for (int k = 0; k < kTriSmallS - 1; k++) {
        if (k < s - 1) {
#pragma unroll
          for (int i = k + 1; i < kTriSmallS; i++)
            if (i < s) x[i] = sub_s(x[i], mul_s(D[i + k * s], x[k]));
        }
      }
    } else {
#pragma unroll
      for (int k = kTriSmallS - 1; k >= 0; k--) {
        if (k < s) {
          const T ukk = D[k + k * s];
          if (is_zero(ukk) && lane == 0) set_error(S.err, DEV_ZERO_PIVOT, S.sn_first[K] + k);
          x[k] = div_s(x[k], ukk);
#pragma unroll
          for (int i = 0; i < k; i++) x[i] = sub_s(x[i], mul_s(D[i + k * s], x[k]));
        }
      }
    }
    if (lane < s) {
      T* W = out + wofs[t] + (int64_t)lane * s;
#pragma unroll
      for (int i = 0; i < kTriSmallS; i++)
        if (i < s) W[i] = x[i];
    }
  }
}

// Row-panel product C(m, n) = alpha sum_k op(A)(m, k) op(B)(k, n) (+ beta
// C, or atomically added), one thread per row m and columns j0 .. j0 +
// NW - 1, k over the task's K chunk [kb, ke).  TRI = 1 (op(B) lower
// triangular, zero for k < n) or 2 (upper, zero for k > n): square op(B);
// in the diagonal block (k in [j0, j0 + NW)) only the triangle is
// multiplied, the other k of the chunk run over all NW columns.  An upper
// op(A) (GEMM_TRI_UPPER_A, with a lower op(B)) starts every warp at its
// first row.  Lanes past M read row M - 1 and columns past N read column
// N - 1 (in bounds; never stored).  FP64 throughput is the bound: the loads
// of op(B) are warp-uniform, those of A coalesced along m (or, transposed,
// one row per lane reused from L1).
template <typename T, int NW, int TRI>
__device__ __forceinline__ void rows_task(const GemmDesc& d, int m, int warp_m0, int j0, int kb,
                                          int ke) {
  const T* __restrict__ B = (const T*)d.B;
  const int mm = min(m, d.M - 1);
  const T* __restrict__ Ar = (const T*)d.A + (d.transA ? (int64_t)mm * d.lda : (int64_t)mm);
  const int64_t ak = d.transA ? 1 : d.lda;
  const int nlast = d.N - 1;
  const int64_t sk = d.transB ? d.ldb : 1, sn = d.transB ? 1 : d.ldb;
  auto bval = [&](int k, int q) { return B[(int64_t)k * sk + (int64_t)min(j0 + q, nlast) * sn]; };
  T acc[NW];
#pragma unroll
  for (int q = 0; q < NW; q++) acc[q] = sc_zero(T());
  // k in [k0, k1) over all NW columns, the operands of k + 1 loaded while
  // those of k are multiplied (a warp alone on its FP64 unit stays busy)
  auto full_range = [&](int k0, int k1) {
    if (k0 >= k1) return;
    T an = Ar[(int64_t)k0 * ak], bn[NW];
#pragma unroll
    for (int q = 0; q < NW; q++) bn[q] = bval(k0, q);
    for (int k = k0; k < k1; k++) {
      const T a = an;
      T b[NW];
#pragma unroll
      for (int q = 0; q < NW; q++) b[q] = bn[q];
      if (k + 1 < k1) {
        an = Ar[(int64_t)(k + 1) * ak];
#pragma unroll
        for (int q = 0; q < NW; q++) bn[q] = bval(k + 1, q);
      }
#pragma unroll
      for (int q = 0; q < NW; q++) acc[q] = fma_s(a, b[q], acc[q]);
    }
  };
  if (TRI == 1) {
    const int kstart = max(kb, (d.tri & GEMM_TRI_UPPER_A) ? max(j0, warp_m0) : j0);
#pragma unroll
    for (int kk = 0; kk < NW; kk++) {
      const int k = j0 + kk;
      if (k < kstart || k >= ke) continue;
      const T a = Ar[(int64_t)k * ak];
#pragma unroll
      for (int q = 0; q <= kk; q++) acc[q] = fma_s(a, bval(k, q), acc[q]);
    }
    full_range(max(j0 + NW, kstart), ke);
  } else if (TRI == 2) {
    full_range(kb, min(j0, ke));
#pragma unroll
    for (int kk = 0; kk < NW; kk++) {
      const int k = j0 + kk;
      if (k < kb || k >= ke) continue;
      const T a = Ar[(int64_t)k * ak];
#pragma unroll
      for (int q = kk; q < NW; q++) acc[q] = fma_s(a, bval(k, q), acc[q]);
    }
  } else {
    full_range(kb, ke);
  }
  if (m >= d.M) return;
  T* __restrict__ C = (T*)d.C + m;
#pragma unroll
  for (int q = 0; q < NW; q++) {
    const int n = j0 + q;
    if (n >= d.N) break;
    T v = scale_s(acc[q], d.alpha);
    if (d.atomic) {
      atomic_add_s(C + (int64_t)n * d.ldc, v);
      continue;
    }
    if (d.beta != 0.0) v = add_s(v, scale_s(C[(int64_t)n * d.ldc], d.beta));
    C[(int64_t)n * d.ldc] = v;
  }
}

template <typename T, int TRI>
__device__ __forceinline__ void rows_dispatch(const GemmDesc& d, int nw, int m, int warp_m0, int j0,
                                              int kb, int ke) {
  if (nw == 4)
    rows_task<T, 4, TRI>(d, m, warp_m0, j0, kb, ke);
  else
    rows_task<T, 8, TRI>(d, m, warp_m0, j0, kb, ke);
}

// Tasks {d, row block, column chunk, NW + 16 x K chunk index}
template <typename T>
__global__ void __launch_bounds__(kRowsBlock)
rows_gemm_kernel(const GemmDesc* __restrict__ descs, const GemmTask* __restrict__ tasks, int ntasks) {
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const GemmTask task = tasks[t];
    const GemmDesc d = descs[task.d];
    const int m = task.tm * kRowsBlock + (int)threadIdx.x;
    const int warp_m0 = m & ~31;
    if (warp_m0 >= d.M) continue;  // whole warp past the last row
    const int j0 = task.tn * kRowsChunk, nw = task.ks & 15, kc = task.ks >> 4;
    const int kchunk = (d.K + d.ksplit - 1) / d.ksplit;
    const int kb = kc * kchunk, ke = min(d.K, kb + kchunk);
    if (d.tri & GEMM_TRI_LOWER_B)
      rows_dispatch<T, 1>(d, nw, m, warp_m0, j0, kb, ke);
    else if (d.tri & GEMM_TRI_UPPER_B)
      rows_dispatch<T, 2>(d, nw, m, warp_m0, j0, kb, ke);
    else
      rows_dispatch<T, 0>(d, nw, m, warp_m0, j0, kb, ke);
  }
}

template <typename T, int BM, int BN, int BK>
void gemm_launch_t(const GemmDesc* descs, const GemmTask* tasks, int ntasks, int grid,
                   cudaStream_t st) {
  if (ntasks <= 0) return;
  gemm_kernel<T, BM, BN, BK><<<grid, kThreads, 0, st>>>(descs, tasks, ntasks);
}

}  // namespace

int gemm_tile_m(int dtype, int cfg) {
  if (cfg == GEMM_128x64) return dtype == DT_F64 ? 128 : 64;
  if (cfg == GEMM_32x32) return 32;
  return dtype == DT_F64 ? 64 : 32;
}
int gemm_tile_n(int dtype, int cfg) {
  if (cfg == GEMM_128x64) return dtype == DT_F64 ? 64 : 32;
  if (cfg == GEMM_32x32) return dtype == DT_F64 ? 32 : 16;
  return dtype == DT_F64 ? 64 : 32;
}

void launch_gemm(int dtype, int cfg, const GemmDesc* descs, const GemmTask* tasks, int ntasks,
                 int grid, cudaStream_t st) {
  if (cfg == GEMM_ROWS) {
    if (ntasks <= 0) return;
    if (dtype == DT_F64)
      rows_gemm_kernel<double><<<grid, kRowsBlock, 0, st>>>(descs, tasks, ntasks);
    else
      rows_gemm_kernel<cdouble><<<grid, kRowsBlock, 0, st>>>(descs, tasks, ntasks);
    return;
  }
  if (dtype == DT_F64) {
    switch (cfg) {
      case GEMM_32x32: gemm_launch_t<double, 32, 32, 16>(descs, tasks, ntasks, grid, st); break;
      case GEMM_128x64: gemm_launch_t<double, 128, 64, 8>(descs, tasks, ntasks, grid, st); break;
      default: gemm_launch_t<double, 64, 64, 16>(descs, tasks, ntasks, grid, st); break;
    }
  } else {
    switch (cfg) {
      case GEMM_32x32: gemm_launch_t<cdouble, 32, 16, 16>(descs, tasks, ntasks, grid, st); break;
      case GEMM_128x64: gemm_launch_t<cdouble, 64, 32, 8>(descs, tasks, ntasks, grid, st); break;
      default: gemm_launch_t<cdouble, 32, 32, 16>(descs, tasks, ntasks, grid, st); break;
    }
  }
}

void launch_lu_panel(int dtype, const SymDev& S, void* store, const SnTask* tasks, int ntasks,
                     cudaStream_t st) {
  if (ntasks <= 0) return;
  if (dtype == DT_F64)
    lu_panel_kernel<double><<<ntasks, kThreads, 0, st>>>(S, (double*)store, tasks, ntasks);
  else
    lu_panel_kernel<cdouble><<<ntasks, kThreads, 0, st>>>(S, (cdouble*)store, tasks, ntasks);
}

cudaError_t prepare_dense_kernels(int, int) { return cudaSuccess; }

namespace {
// FP64 pipe throughput: kPeakChains independent fused multiply-add chains
// per thread (enough to hide the pipe's latency), `iters` rounds; the sum is
// stored so that nothing is optimised away.
constexpr int kPeakChains = 8;
__global__ void __launch_bounds__(kThreads)
fp64_peak_kernel(double* out, int iters, double a, double b) {
  double x[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; j++) x[j] = threadIdx.x * 1e-3 + j;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < kPeakChains; j++) x[j] = fma(x[j], a, b);
  }
  double sum = 0.0;
#pragma unroll
  for (int j = 0; j < kPeakChains; j++) sum += x[j];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = sum;
}
}  // namespace

int fp64_peak_grid(int sms) { return sms * 8; }

// flops of one launch of the FP64 peak loop over `grid` CTAs
double launch_fp64_peak(double* out, int grid, int iters, cudaStream_t st) {
  fp64_peak_kernel<<<grid, kThreads, 0, st>>>(out, iters, 0.999999, 1e-7);
  return 2.0 * kPeakChains * (double)iters * (double)grid * kThreads;
}

void launch_tri_inv(int dtype, const SymDev& S, const void* store, void* out,
                    const int64_t* wofs, const SnTask* tasks, int ntasks, int, int small,
                    cudaStream_t st) {
  if (ntasks <= 0) return;
  // one task (or one warp's task) per CTA: the launches often run on a
  // low-priority stream, and short CTAs let the sweep's CTAs in between
  if (small) {
    const int warps = kThreads / 32;
    const int grid = (ntasks + warps - 1) / warps;
    if (dtype == DT_F64)
      tri_inv_small_kernel<double><<<grid, kThreads, 0, st>>>(S, (const double*)store,
                                                              (double*)out, wofs, tasks, ntasks);
    else
      tri_inv_small_kernel<cdouble><<<grid, kThreads, 0, st>>>(S, (const cdouble*)store,
                                                               (cdouble*)out, wofs, tasks, ntasks);
    return;
  }
  const int grid = ntasks;
  if (dtype == DT_F64)
    tri_inv_kernel<double><<<grid, kThreads, 0, st>>>(S, (const double*)store, (double*)out, wofs,
                                                      tasks, ntasks);
  else
    tri_inv_kernel<cdouble><<<grid, kThreads, 0, st>>>(S, (const cdouble*)store, (cdouble*)out,
                                                       wofs, tasks, ntasks);
}

}  // namespace pselinv
