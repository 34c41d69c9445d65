// Split-precision (Ozaki-scheme) products on the 5th-generation tensor
// cores: the bulk GEMMs of Algorithm 1 steps 3-5 computed as sums of FP16
// slice products accumulated exactly in FP32 and recombined in 64-bit
// integers, then scaled back to FP64.
//
// Slicing.  Each row r of an operand X (rows = the M or N dimension, columns
// = the contracted K dimension) is scaled by 2^-e_r with e_r the binary
// exponent of max_k |X(r,k)| (so |x| 2^-e_r < 1), rounded to the fixed-point
// integer Q = rint(x 2^{7S - e_r}) (|Q| <= 2^{7S}), and Q is written in
// balanced base 128:  Q = sum_s a_s 128^{S-1-s},  |a_s| <= 64 for s >= 1,
// |a_0| <= 128, so every digit is an integer held exactly by FP16 and
//   x = 2^e_r sum_s a_s 2^{-7(s+1)} + O(2^{e_r - 7S - 1}).
// The conversion works on the bit pattern of x with integer operations only
// (the FP64 pipe of GB300 is too slow to slice with).
// Products.  For slice pairs (s, t) with s + t = d <= S-1, the products
// a_s(A) b_t(B) are summed in one FP32 tensor-memory accumulator per weight
// d over 512 values of K: one value of K adds at most 2^14 (d = 0, 1) and at
// most 2 x 2^13 + (d-1) 2^12 <= 2^15 (d <= 5) to an accumulator, so every
// partial sum stays an integer of magnitude <= 2^24, exact in FP32.  After
// each 512-wide chunk the S accumulators are drained into a 64-bit integer
// per output held in tensor memory,
//   T += sum_d P_d 2^{7(S-1-d)}   (|T| < 31 x 2^58.01 < 2^63 for K <= 31 x 512),
// and at the end C = T 2^{e_r(A) + e_c(B) - 14 - 7(S-1)} in FP64.
// The only rounding is the slice truncation and the final int64 -> FP64
// conversion.
//
// Layouts.  A slice set stores, for every slice s, every 64-row block and
// every 32-wide K block, a 4 KB tile in the tcgen05 canonical K-major layout
// without swizzle: 8x16-byte core matrices, core (row group g, k group kg) at
// byte (g * 4 + kg) * 128.  Two consecutive 64-row tiles form the 128-row A
// operand (LBO = 128 B along K, SBO = 512 B along M); one tile is the B
// operand of a 64-column output tile.
#include <cuda_fp16.h>

#include "device.cuh"

namespace pselinv {

namespace {

constexpr int kSliceThreads = 256;
constexpr int kTileBytes = 4096;  // 64 rows x 32 K x 2 bytes
constexpr unsigned long long kWaitBudgetNs = 2000000000ull;  // 2 s per bounded wait
constexpr int kChunk = 16;  // 32-wide K blocks per exact accumulation chunk (512 values)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------------------
// slicing
// ---------------------------------------------------------------------------
// |x| as the bit pattern of a non-negative double (orders like the value)
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
// e with max < 2^e (the frexp exponent) from the bits of a non-negative max;
// zero and subnormal maxima give 0 (those rows are sliced to zero)
__device__ __forceinline__ int exp_of_max(unsigned long long bits) {
  const int E = (int)(bits >> 52);
  return E == 0 ? 0 : E - 1022;
}
// |Q| = rint(|x| 2^{sh0}) (|Q| <= 2^{7S}, from the bits of x) split at bit
// B: lo = |Q| mod 2^B and hi = |Q| >> B, returned as exact floats that
// carry the sign of x (both below 2^23 in magnitude)
__device__ __forceinline__ void fixed_point_split(double x, int sh0, int B, float& lo, float& hi) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  const int r = 1075 - E - sh0;  // |x| 2^{sh0} = M 2^{-r}
  unsigned long long q = 0;
  if (E != 0 && r < 54) {  // r >= 54: below one half
    const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int rr = r < 1 ? 1 : r;  // r > 7 for every |x| below 2^e
    q = (M + (1ull << (rr - 1))) >> rr;
  }
  const uint32_t ql = (uint32_t)q & ((1u << B) - 1u);
  const uint32_t qh = (uint32_t)(q >> B);
  // 2^23 + k has the bits 0x4B000000 | k (k < 2^23)
  const float sg = (long long)b < 0 ? -1.0f : 1.0f;
  lo = __fmaf_rn(__uint_as_float(0x4B000000u | ql), sg, -8388608.0f * sg);
  hi = __fmaf_rn(__uint_as_float(0x4B000000u | qh), sg, -8388608.0f * sg);
}

// One balanced base-128 digit of an integer-valued float v (|v| < 2^22):
// v = 128 t + a with t = rint(v / 128) (ties to even) and |a| <= 64; v
// becomes t.  All three operations are exact.
__device__ __forceinline__ float digit_step(float& v) {
  constexpr float kRound = 12582912.0f;  // 1.5 * 2^23: adding it rounds to an integer
  const float t = __fsub_rn(__fmaf_rn(v, 0.0078125f, kRound), kRound);
  const float a = __fmaf_rn(-128.0f, t, v);
  v = t;
  return a;
}

// Work item of the slicing kernels: thread t of a task covers row
// rl = (ci / 4) * 8 + rr and the 8 values of K group kg = ci % 4 of one
// 32-wide K block (ci = t / 8, rr = t % 8), i.e. bytes [16t, 16t+16) of the
// block's 4 KB tile in every slice.  One task = one 64-row block and
// kSliceSpan consecutive K blocks; the values are loaded straight into
// registers (each lane reads its 8 values; lanes of a warp cover 8 rows x 4
// groups).
constexpr int kSliceSpan = 2;

// 8 consecutive values X(r, k0 .. k0+7) of the slice set's K range (for a
// complex source: real parts in the first half of the range, imaginary
// parts in the second)
__device__ __forceinline__ void load8(const SliceDesc& d, int r, int k0, double (&x)[8]) {
  const double* __restrict__ src = d.src;
  int part = 0;
  if (d.cplx) {
    const int half = (d.K32 / 2) * 32;
    if (k0 >= half) {
      part = 1;
      k0 -= half;
    }
  }
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int k = k0 + j;
    double v = 0.0;
    if (r < d.R && k < d.Kd) {
      const int64_t idx = d.mode == SLICE_ROWS ? r + (int64_t)k * d.ld : k + (int64_t)r * d.ld;
      v = d.cplx ? src[2 * idx + part] : src[idx];
    }
    x[j] = v;
  }
}

// Row maxima of |X| (bit patterns) of one task, accumulated with atomicMax
// into d.maxbits (zeroed beforehand).
__device__ __forceinline__ void slice_max_task(const SliceDesc& d, const SliceTask& task, int tid) {
  const int ci = tid >> 3, rr = tid & 7;
  const int rl = (ci >> 2) * 8 + rr, kg = ci & 3;
  const int r = task.rb * 64 + rl;
  unsigned long long m = 0;
  const int kb1 = min(d.K32, (task.kc + 1) * kSliceSpan);
  for (int kb = task.kc * kSliceSpan; kb < kb1; kb++) {
    double x[8];
    load8(d, r, kb * 32 + kg * 8, x);
#pragma unroll
    for (int j = 0; j < 8; j++) m = max(m, abs_bits(x[j]));
  }
  // the 4 lanes sharing a row are tid ^ 8, ^ 16 (same rr, kg = 0..3 inside a warp)
  m = max(m, __shfl_xor_sync(0xffffffffu, m, 8));
  m = max(m, __shfl_xor_sync(0xffffffffu, m, 16));
  if (kg == 0 && r < d.R && m) atomicMax(d.maxbits + r, m);
}

// The S balanced base-128 digits of 8 values x of one row with exponent e,
// written as the 16 bytes [16 tid, 16 tid + 16) of the 4 KB tile of every
// slice at `dst` (slices `slice_stride` halves apart).  Q = rint(x 2^{7S-e})
// (|Q| <= 2^{7S}) is split once into its low 7 L bits (L = S / 2 digits)
// and the rest, both exact floats, so that the digits come from FP32
// arithmetic: the low digits leave a carry of -1, 0 or 1 into the high
// part.  Digits below the top one lie in [-64, 64]; the top one is what
// remains (|a| <= 128, as |Q| <= 2^{7S} and the lower digits sum to less
// than half a top unit), and sum_s a_s 128^{S-1-s} = Q exactly.
template <int S>
__device__ __forceinline__ void write_digits_s(const double (&x)[8], int e, __half* dst,
                                               int64_t slice_stride) {
  constexpr int L = S / 2;
  const int sh0 = 7 * S - e;
  float lo[8], hi[8];
#pragma unroll
  for (int j = 0; j < 8; j++) fixed_point_split(x[j], sh0, 7 * L, lo[j], hi[j]);
  // from the least significant slice upwards
#pragma unroll
  for (int s = S - 1; s >= 0; s--) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      if (s >= S - L) {
        a[j] = digit_step(lo[j]);
        if (s == S - L) hi[j] += lo[j];  // carry of the low digits (exact)
      } else {
        a[j] = s > 0 ? digit_step(hi[j]) : hi[j];
      }
    }
    uint4 w;
    __half2 h0 = __floats2half2_rn(a[0], a[1]), h1 = __floats2half2_rn(a[2], a[3]);
    __half2 h2 = __floats2half2_rn(a[4], a[5]), h3 = __floats2half2_rn(a[6], a[7]);
    w.x = *reinterpret_cast<uint32_t*>(&h0);
    w.y = *reinterpret_cast<uint32_t*>(&h1);
    w.z = *reinterpret_cast<uint32_t*>(&h2);
    w.w = *reinterpret_cast<uint32_t*>(&h3);
    *reinterpret_cast<uint4*>(dst + s * slice_stride) = w;
  }
}
__device__ __forceinline__ void write_digits(const double (&x)[8], int e, int S, __half* dst,
                                             int64_t slice_stride) {
  if (S == 6)
    write_digits_s<6>(x, e, dst, slice_stride);
  else if (S == 5)
    write_digits_s<5>(x, e, dst, slice_stride);
  else
    write_digits_s<4>(x, e, dst, slice_stride);
}

// Slices of one task (see the work item above); exponents from d.maxbits.
__device__ __forceinline__ void slice_task(const SliceDesc& d, const SliceTask& task, int tid) {
  const int ci = tid >> 3, rr = tid & 7;
  const int rl = (ci >> 2) * 8 + rr, kg = ci & 3;
  const int r = task.rb * 64 + rl;
  const int e = r < d.R ? exp_of_max(d.maxbits[r]) : 0;
  if (task.kc == 0 && kg == 0 && r < d.R) d.exps[r] = e;
  const int64_t slice_stride = (int64_t)d.R64 * d.K32 * (kTileBytes / 2);  // halves
  const int kb1 = min(d.K32, (task.kc + 1) * kSliceSpan);
  for (int kb = task.kc * kSliceSpan; kb < kb1; kb++) {
    double x[8];
    load8(d, r, kb * 32 + kg * 8, x);
    write_digits(x, e, d.S,
                 d.out + ((int64_t)task.rb * d.K32 + kb) * (kTileBytes / 2) + tid * 8,
                 slice_stride);
  }
}

__global__ void __launch_bounds__(kSliceThreads)
slice_max_kernel(const SliceDesc* __restrict__ descs, const SliceTask* __restrict__ tasks, int ntasks) {
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SliceTask task = tasks[t];
    slice_max_task(descs[task.d], task, threadIdx.x);
  }
}

__global__ void __launch_bounds__(kSliceThreads)
slice_kernel(const SliceDesc* __restrict__ descs, const SliceTask* __restrict__ tasks, int ntasks) {
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SliceTask task = tasks[t];
    slice_task(descs[task.d], task, threadIdx.x);
  }
}

// ---------------------------------------------------------------------------
// G = Ainv(R_K, R_K) sliced straight from the ancestors' blocks
// ---------------------------------------------------------------------------
// A task stages one 64 x 64 tile of G in shared memory, reading each entry
// once through the block index map (Algorithm 1's gather of Ainv_CC): the
// entries on or below the block diagonal down the columns of the diagonal
// blocks and L panels of the ancestors (lanes along the rows), the ones
// above it along the rows of their U^T panels (lanes along the columns).
// Per column and per row of the tile, the storage column and the relative
// index list are looked up once, so an entry costs one index load and one
// value load.  The maxima pass then accumulates the tile's row and column
// maxima; the slicing pass writes the tile's slices in both layouts that
// steps 3 and 5 read (G by rows and G by columns), so G is never written in
// FP64.  Tasks past the G tiles are ordinary slice tasks (the panels of the
// same level).
constexpr int kGT = 64;        // G tile side
constexpr int kGTPad = kGT + 1;

template <typename T>
__device__ __forceinline__ unsigned long long abs_bits_max(T v);
template <>
__device__ __forceinline__ unsigned long long abs_bits_max<double>(double v) {
  return abs_bits(v);
}
template <>
__device__ __forceinline__ unsigned long long abs_bits_max<cdouble>(cdouble v) {
  return max(abs_bits(v.x), abs_bits(v.y));
}
__device__ __forceinline__ double part_of(double v, int) { return v; }
__device__ __forceinline__ double part_of(cdouble v, int part) { return part ? v.y : v.x; }

template <typename T>
constexpr size_t gslice_smem() {
  // tile + per column (diag base, L base, relative base: int64; block: int)
  // + per row (U^T base, relative base: int64; block: int)
  return (size_t)kGT * kGTPad * sizeof(T) + (size_t)kGT * (5 * 8 + 2 * 4);
}

template <typename T, bool MAXIMA>
__global__ void __launch_bounds__(kSliceThreads, 4)
gslice_kernel(SymDev S, const T* __restrict__ store, const SliceDesc* __restrict__ descs,
              const GTileTask* __restrict__ gtasks, int ngt,
              const SliceTask* __restrict__ stasks, int nst, unsigned long long* rcmax) {
  extern __shared__ __align__(16) unsigned char gs_raw[];
  T* tile = reinterpret_cast<T*>(gs_raw);  // tile[pl * kGTPad + ql]
  int64_t* cdiag = reinterpret_cast<int64_t*>(gs_raw + (size_t)kGT * kGTPad * sizeof(T));
  int64_t* cpan = cdiag + kGT;
  int64_t* crel = cpan + kGT;
  int64_t* rpan = crel + kGT;
  int64_t* rrel = rpan + kGT;
  int* cblk = reinterpret_cast<int*>(rrel + kGT);
  int* rblk = cblk + kGT;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int t = blockIdx.x; t < ngt + nst; t += gridDim.x) {
    if (t >= ngt) {
      const SliceTask task = stasks[t - ngt];
      if (MAXIMA)
        slice_max_task(descs[task.d], task, tid);
      else
        slice_task(descs[task.d], task, tid);
      continue;
    }
    const GTileTask task = gtasks[t];
    const int K = task.K;
    // G_K = Ainv(R_U(K), R_L(K)): cu rows (positions p), cl columns (q);
    // R_U = R_L = R_K for a structurally symmetric handle
    const int cl = S.sn_c[K], cu = S.general ? S.sn_cu[K] : cl;
    const int64_t rb = S.rows_ptr[K], rbU = S.general ? S.urows_ptr[K] : rb;
    const int64_t io = (int64_t)task.inst * S.storage;
    const int p0 = task.tp * kGT, q0 = task.tq * kGT;
    // per-column and per-row storage bases of the tile (precomputed per
    // position: independent loads, no chain through the block maps); the
    // supernode of each row and column decides where an entry lies
    if (tid < kGT) {
      const int q = q0 + tid;
      if (q < cl) {
        cdiag[tid] = io + S.col_diag[rb + q];
        cpan[tid] = io + S.col_pan[rb + q];
        crel[tid] = S.col_rel[rb + q];
        cblk[tid] = S.col_sn[rb + q];
      } else {
        cblk[tid] = 0x7FFFFFFF;
      }
    } else if (tid < 2 * kGT) {
      const int pl = tid - kGT, p = p0 + pl;
      if (p < cu) {
        rpan[pl] = io + S.row_pan[rbU + p];
        rrel[pl] = S.row_rel[rbU + p];
        rblk[pl] = S.row_sn[rbU + p];
      } else {
        rblk[pl] = -1;
      }
    }
    __syncthreads();
    constexpr int kPer = kGT * kGT / kSliceThreads / 2;  // entries per thread and round
    // entries whose row lies in the column's supernode or later: lanes along
    // p (down a column); in two rounds, all index loads of a round first,
    // then all its value loads
#pragma unroll 1
    for (int round = 0; round < 2; round++) {
      int rel[kPer];
      bool use[kPer];
#pragma unroll
      for (int ii = 0; ii < kPer; ii++) {
        const int i = round * kPer + ii;
        const int ql = warp + 8 * (i >> 1), pl = lane + 32 * (i & 1);
        const int p = p0 + pl, q = q0 + ql;
        use[ii] = p < cu && q < cl && rblk[pl] >= cblk[ql];
        int64_t ri = crel[ql] + p;
        if (S.check && use[ii] && (ri < 0 || ri >= S.relidx_size)) {
          set_error(S.err, DEV_CHECK, K);
          use[ii] = false;
        }
        rel[ii] = use[ii] ? S.relidx[ri] : 0;
      }
      T v[kPer];
#pragma unroll
      for (int ii = 0; ii < kPer; ii++) {
        const int i = round * kPer + ii;
        const int ql = warp + 8 * (i >> 1), pl = lane + 32 * (i & 1);
        const int64_t slot = (rblk[pl] == cblk[ql] ? cdiag[ql] : cpan[ql]) + rel[ii];
        if (S.check && use[ii] && (slot < io || slot >= io + S.storage)) {
          set_error(S.err, DEV_CHECK, K);
          use[ii] = false;
        }
        v[ii] = use[ii] ? store[slot] : sc_zero(T());
      }
#pragma unroll
      for (int ii = 0; ii < kPer; ii++) {
        const int i = round * kPer + ii;
        const int ql = warp + 8 * (i >> 1), pl = lane + 32 * (i & 1);
        if (p0 + pl >= cu || q0 + ql >= cl || rblk[pl] >= cblk[ql])  // upper pass writes the rest
          tile[pl * kGTPad + ql] = v[ii];
      }
    }
    // the others: lanes along q (down a column of a panel of the row's supernode)
#pragma unroll 1
    for (int round = 0; round < 2; round++) {
      int rel[kPer];
      bool use[kPer];
#pragma unroll
      for (int ii = 0; ii < kPer; ii++) {
        const int i = round * kPer + ii;
        const int pl = warp + 8 * (i >> 1), ql = lane + 32 * (i & 1);
        const int p = p0 + pl, q = q0 + ql;
        use[ii] = p < cu && q < cl && rblk[pl] < cblk[ql];
        const int64_t ri = rrel[pl] + q;
        if (S.check && use[ii] && (ri < 0 || ri >= S.relidx_size)) {
          set_error(S.err, DEV_CHECK, K);
          use[ii] = false;
        }
        rel[ii] = use[ii] ? S.relidx[ri] : 0;
      }
      T v[kPer];
#pragma unroll
      for (int ii = 0; ii < kPer; ii++) {
        const int i = round * kPer + ii;
        const int pl = warp + 8 * (i >> 1);
        const int64_t slot = rpan[pl] + rel[ii];
        if (S.check && use[ii] && (slot < io || slot >= io + S.storage)) {
          set_error(S.err, DEV_CHECK, K);
          use[ii] = false;
        }
        v[ii] = use[ii] ? store[slot] : sc_zero(T());
      }
#pragma unroll
      for (int ii = 0; ii < kPer; ii++) {
        const int i = round * kPer + ii;
        const int pl = warp + 8 * (i >> 1), ql = lane + 32 * (i & 1);
        if (p0 + pl < cu && q0 + ql < cl && rblk[pl] < cblk[ql]) tile[pl * kGTPad + ql] = v[ii];
      }
    }
    __syncthreads();
    const SliceDesc& dr = descs[task.dr];
    // the running row / column maxima of this instance
    unsigned long long* rmax = rcmax + (int64_t)task.inst * 2 * S.n;
    unsigned long long* cmax = rmax + S.n;
    const int32_t* ridx = (S.general ? S.urows : S.lrows) + rbU;  // global row of position p
    const int32_t* cidx = S.lrows + rb;                              // global column of q
    if (MAXIMA) {
      // row maxima, then column maxima: four threads (a quarter of the
      // tile's width each, neighbours in one warp) per row / column
      const int line = tid >> 2, part = tid & 3;
      unsigned long long m = 0;
      for (int i = 0; i < kGT / 4; i++)
        m = max(m, abs_bits_max(tile[line * kGTPad + part * (kGT / 4) + i]));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 1));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 2));
      if (part == 0 && p0 + line < cu && m) atomicMax(rmax + ridx[p0 + line], m);
      m = 0;
      for (int i = 0; i < kGT / 4; i++)
        m = max(m, abs_bits_max(tile[(part * (kGT / 4) + i) * kGTPad + line]));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 1));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 2));
      if (part == 0 && q0 + line < cl && m) atomicMax(cmax + cidx[q0 + line], m);
    } else {
      // work item of the slicing: row rl, 8 values of K group kg of a 32-wide K block
      const int ci = tid >> 3, rr = tid & 7;
      const int rl = (ci >> 2) * 8 + rr, kg = ci & 3;
      constexpr int kParts = sizeof(T) == 16 ? 2 : 1;
      for (int layout = 0; layout < 2; layout++) {
        if (layout == 1 && task.dc < 0) break;
        // layout 0: G by rows (rows p, K = q); layout 1: G by columns
        const SliceDesc& d = layout == 0 ? dr : descs[task.dc];
        const int r0 = layout == 0 ? p0 : q0;   // rows of this layout's tile
        const int kq0 = layout == 0 ? q0 : p0;  // its K offset
        const int nrows = layout == 0 ? cu : cl, nk = layout == 0 ? cl : cu;
        const int k32c = (nk + 31) / 32;  // K blocks of one part
        const int rblk64 = r0 / 64;
        const int r = r0 + rl;
        // G by rows: rows of Ainv; by columns: its columns (a symmetric G,
        // sliced by rows only, takes the larger of both)
        unsigned long long mb = 0;
        if (r < nrows) {
          mb = layout == 0 ? rmax[ridx[r]] : cmax[cidx[r]];
          if (task.dc < 0) mb = max(mb, cmax[cidx[r]]);
        }
        const int e = r < nrows ? exp_of_max(mb) : 0;
        if (kq0 == 0 && kg == 0 && r < nrows) d.exps[r] = e;
        const int64_t slice_stride = (int64_t)d.R64 * d.K32 * (kTileBytes / 2);
        for (int kbl = 0; kbl < kGT / 32; kbl++) {
          const int kb = kq0 / 32 + kbl;
          if (kb >= k32c) break;
          for (int part = 0; part < kParts; part++) {
            double x[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
              const int kl = kbl * 32 + kg * 8 + j;
              const T v = layout == 0 ? tile[rl * kGTPad + kl] : tile[kl * kGTPad + rl];
              x[j] = part_of(v, part);
            }
            const int kbp = kb + part * k32c;
            write_digits(x, e, d.S,
                         d.out + ((int64_t)rblk64 * d.K32 + kbp) * (kTileBytes / 2) + tid * 8,
                         slice_stride);
          }
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// tcgen05 helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  // K-major, no swizzle: LBO (K direction) = 128 B, SBO (M/N direction) = 512 B
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// kind::f16, FP16 x FP16 -> FP32, both operands K-major, M = 128, N = 64
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr uint32_t kIdescNegA = kIdesc | (1u << 13);  // D += (-A) B
// the same with N = 128: two B slices tb, tb + 1 (adjacent 4 KB tiles, so
// one operand of 128 rows at the same 512-byte row-group stride) into the
// adjacent accumulators of weights s + tb and s + tb + 1, A read once
constexpr uint32_t kIdescN128 =
    (1u << 4) | ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr uint32_t kIdescN128NegA = kIdescN128 | (1u << 13);

__device__ __forceinline__ void mma_f16(uint32_t dt, uint64_t a, uint64_t b, uint32_t acc,
                                        uint32_t idesc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// the same with A from tensor memory (128 lanes = rows, 8 columns = K 16)
__device__ __forceinline__ void mma_f16_ta(uint32_t dt, uint32_t at, uint64_t b, uint32_t acc,
                                           uint32_t idesc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dt),
      "r"(at), "l"(b), "r"(idesc), "r"(acc));
}
// 128 rows x 256 bits (K 16 of FP16) from shared memory (canonical K-major
// layout of the descriptor) into tensor memory: row i -> lane i
__device__ __forceinline__ void tmem_cp_128x256b(uint32_t taddr, uint64_t sdesc) {
  asm volatile("tcgen05.cp.cta_group::1.128x256b [%0], %1;" ::"r"(taddr), "l"(sdesc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait on a phase parity: false once `budget_ns` of wall-clock time
// has passed without the phase completing
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity,
                                          unsigned long long budget_ns = kWaitBudgetNs) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > budget_ns) return false;
  }
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
        "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
        "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// v * 2^e as the nearest double (ties to even), built from the integer bits
// without FP64 arithmetic; results below the normal range flush to zero.
__device__ __forceinline__ double scaled_int_to_double(long long v, int e, bool negate) {
  if (v == 0) return 0.0;
  unsigned long long sign = (v < 0) != negate ? (1ull << 63) : 0ull;
  unsigned long long u = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll(u);
  u <<= lz;  // leading one at bit 63
  unsigned long long m = u >> 11;
  const unsigned long long r = u & 0x7FFull;
  if (r > 0x400ull || (r == 0x400ull && (m & 1ull))) m++;
  int E = e + 63 - lz + 1023;
  if (m == (1ull << 53)) {
    m >>= 1;
    E++;
  }
  if (E <= 0) return 0.0;
  if (E >= 2047) return __longlong_as_double((long long)(sign | (0x7FFull << 52)));
  return __longlong_as_double((long long)(sign | ((unsigned long long)E << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]),
      "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]),
      "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// sliced GEMM: one 128 x 64 output tile (and one K range) per task,
// persistent CTAs with three roles
//   warp 8 (one lane): bulk copies of the slice tiles into a 2-stage ring,
//   warp 9 (one lane): the tcgen05 MMAs of every stage into the S
//     accumulators; a commit frees the stage, another marks a chunk done,
//   warps 0-7: drain each finished chunk (warp w owns TMEM lanes = output
//     rows 32 (w % 4) .. + 31 and the 32 output columns of half w / 4), hand
//     the accumulators back, add the chunk into the 64-bit totals and,
//     after the last chunk, write the outputs while the MMAs of the next
//     task already run.
// ---------------------------------------------------------------------------
// ring depth: three stages (216 KB for S = 6) hide the copy latency behind
// the paired MMAs of a K block; the tensor-memory-A variant keeps two (its
// totals take 64 KB of shared memory)
template <int S, bool ATMEM>
__host__ __device__ constexpr int oz_stages() {
  return ATMEM || S * 3 * 4096 * 3 > 220 * 1024 ? 2 : 3;
}
constexpr int kOzDrainWarps = 8;
constexpr int kOzThreads = (kOzDrainWarps + 2) * 32;

// K-block range [kb0, kb0 + nkb) of a task (nkb <= 0: nothing to do)
__device__ __forceinline__ void task_range(const OzDesc& d, int ks, int& kb0, int& nkb) {
  int per = (d.K32 + d.ksplit - 1) / d.ksplit;
  per = (per + kChunk - 1) / kChunk * kChunk;
  kb0 = ks * per;
  nkb = min(d.K32, kb0 + per) - kb0;
}

// ATMEM: the A slices go from the stage into tensor memory (tcgen05.cp, K 16
// at a time, two buffers of S x 8 columns after the accumulators) and the
// MMAs read A there, so shared memory serves each A tile once per K half
// instead of once per slice pair; the 64-bit totals then live in shared
// memory (64 KB after the ring) instead of tensor memory.
template <int S, bool ATMEM>
__global__ void __launch_bounds__(kOzThreads, 1)
ozaki_gemm_kernel(const OzDesc* __restrict__ descs, const OzTask* __restrict__ tasks, int ntasks,
                  int* err) {
  constexpr int kAB = S * 2 * kTileBytes;  // A part of a stage (128 rows)
  constexpr int kStage = S * 3 * kTileBytes;
  constexpr int kOzStages = oz_stages<S, ATMEM>();
  constexpr uint32_t kTmemCols = 512;
  static_assert(!ATMEM || S * 64 + 2 * S * 8 <= (int)kTmemCols, "tensor memory budget");
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_full[kOzStages], bar_free[kOzStages], bar_acc_full,
      bar_acc_empty, bar_afree[2];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int i = 0; i < kOzStages; i++) {
      mbar_init(smem_u32(&bar_full[i]), 1);
      mbar_init(smem_u32(&bar_free[i]), 1);
    }
    mbar_init(smem_u32(&bar_acc_full), 1);
    mbar_init(smem_u32(&bar_acc_empty), kOzDrainWarps);  // one arrival per drain warp
    mbar_init(smem_u32(&bar_afree[0]), 1);
    mbar_init(smem_u32(&bar_afree[1]), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  bool ok = true;

  if (warp == kOzDrainWarps) {
    // ---- producer ----
    if (lane == 0) {
      uint32_t g = 0;  // K blocks issued so far (ring position)
      for (int t = blockIdx.x; t < ntasks && ok; t += gridDim.x) {
        const OzTask task = tasks[t];
        const OzDesc* dp = descs + task.d;
        OzDesc d;  // the fields the copies need
        d.A = dp->A; d.B = dp->B; d.A_R64 = dp->A_R64; d.B_R64 = dp->B_R64; d.K32 = dp->K32;
        d.ksplit = dp->ksplit; d.swap_b = dp->swap_b; d.half = dp->half;
        int kb0, nkb;
        task_range(d, task.ks, kb0, nkb);
        const bool a_second = 2 * task.tm + 1 < d.A_R64;
        const uint32_t bytes = (uint32_t)(S * (a_second ? 2 : 1) * kTileBytes + S * kTileBytes);
        const int64_t a_sl = (int64_t)d.A_R64 * d.K32 * kTileBytes;
        const int64_t b_sl = (int64_t)d.B_R64 * d.K32 * kTileBytes;
        const unsigned char* A = reinterpret_cast<const unsigned char*>(d.A);
        const unsigned char* B = reinterpret_cast<const unsigned char*>(d.B);
        for (int i = 0; i < nkb; i++, g++) {
          const int stg = (int)(g % kOzStages);
          const uint32_t u = g / kOzStages;
          if (u > 0 && !mbar_wait(smem_u32(&bar_free[stg]), (u - 1) & 1)) {
            ok = false;
            break;
          }
          if (abort_flag) {
            ok = false;
            break;
          }
          unsigned char* st = smem + stg * kStage;
          const uint32_t fb = smem_u32(&bar_full[stg]);
          mbar_expect_tx(fb, bytes);
          const int kb = kb0 + i;
          const int kbb = d.swap_b ? (kb < d.half ? kb + d.half : kb - d.half) : kb;
          for (int sl = 0; sl < S; sl++) {
            const unsigned char* a0 = A + sl * a_sl + ((int64_t)(2 * task.tm) * d.K32 + kb) * kTileBytes;
            bulk_load(smem_u32(st + sl * 2 * kTileBytes), a0, kTileBytes, fb);
            if (a_second)
              bulk_load(smem_u32(st + sl * 2 * kTileBytes + kTileBytes), a0 + (int64_t)d.K32 * kTileBytes,
                        kTileBytes, fb);
            const unsigned char* b0 = B + sl * b_sl + ((int64_t)task.tn * d.K32 + kbb) * kTileBytes;
            bulk_load(smem_u32(st + kAB + sl * kTileBytes), b0, kTileBytes, fb);
          }
        }
      }
      if (!ok) {
        abort_flag = 1;
        // let the copies already issued land before the CTA exits (bounded)
        for (uint32_t k = g > (uint32_t)kOzStages ? g - kOzStages : 0u; k < g; k++)
          mbar_wait(smem_u32(&bar_full[k % kOzStages]), (k / kOzStages) & 1);
      }
    }
  } else if (warp == kOzDrainWarps + 1) {
    // ---- MMA issue ----
    if (lane == 0) {
      uint32_t g = 0, q = 0;  // K blocks consumed, chunks completed
      uint32_t h16 = 0;       // ATMEM: K halves issued (tensor-memory A buffer ring)
      for (int t = blockIdx.x; t < ntasks && ok; t += gridDim.x) {
        const OzTask task = tasks[t];
        const OzDesc* dp = descs + task.d;
        OzDesc d;  // the fields the MMAs need
        d.K32 = dp->K32; d.ksplit = dp->ksplit; d.half = dp->half; d.neg_half = dp->neg_half;
        int kb0, nkb;
        task_range(d, task.ks, kb0, nkb);
        for (int i = 0; i < nkb; i++, g++) {
          const int stg = (int)(g % kOzStages);
          const bool first = (i % kChunk) == 0;
          const bool last = (i % kChunk == kChunk - 1) || (i == nkb - 1);
          if (first && q > 0 && !mbar_wait(smem_u32(&bar_acc_empty), (q - 1) & 1)) {
            ok = false;
            break;
          }
          if (!mbar_wait(smem_u32(&bar_full[stg]), (g / kOzStages) & 1) || abort_flag) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t st = smem_u32(smem + stg * kStage);
          const bool neg_a = d.neg_half && kb0 + i >= d.half;
          const uint32_t idesc = neg_a ? kIdescNegA : kIdesc;
          const uint32_t idesc2 = neg_a ? kIdescN128NegA : kIdescN128;
          // stage-base descriptors; an offset within shared memory is added
          // to the address field (bits 0-13 hold address >> 4)
          const uint64_t a0 = smem_desc(st), b0 = smem_desc(st + kAB);
          if (ATMEM) {
            bool waited = true;
#pragma unroll 1
            for (int hk = 0; hk < 2; hk++, h16++) {
              const uint32_t x = h16 & 1;
              // the MMAs that read this buffer two halves ago are done
              if (h16 >= 2 && !mbar_wait(smem_u32(&bar_afree[x]), ((h16 - 2) >> 1) & 1)) {
                waited = false;
                break;
              }
              const uint32_t ta = tmem + (uint32_t)(S * 64) + x * (uint32_t)(S * 8);
#pragma unroll
              for (int sa = 0; sa < S; sa++)
                tmem_cp_128x256b(ta + (uint32_t)(sa * 8),
                                 a0 + (uint64_t)((sa * 2 * kTileBytes + hk * 256) >> 4));
#pragma unroll
              for (int sa = 0; sa < S; sa++)
#pragma unroll
                for (int tb = 0; tb < S - sa; tb += 2)
                  mma_f16_ta(tmem + (uint32_t)((sa + tb) * 64), ta + (uint32_t)(sa * 8),
                             b0 + (uint64_t)((tb * kTileBytes + hk * 256) >> 4),
                             (sa == 0 && first && hk == 0) ? 0u : 1u,
                             tb + 1 < S - sa ? idesc2 : idesc);
              mma_commit(smem_u32(&bar_afree[x]));
            }
            if (!waited) {
              // the stage's commit still tracks what was issued, so that the
              // exit below waits for it
              mma_commit(smem_u32(&bar_free[stg]));
              g++;
              ok = false;
              break;
            }
          } else {
            // slice pairs (sa, tb) and (sa, tb + 1) in one N = 128 MMA: 9
            // such and 3 of N = 64 per K 16 for S = 6 instead of 21 of N = 64
            // (an N = 64 MMA is bound by reading its 6 KB of operands from
            // shared memory: 48 cycles against 64 for N = 128's 8 KB and
            // twice the products)
#pragma unroll
            for (int sa = 0; sa < S; sa++)
#pragma unroll
              for (int tb = 0; tb < S - sa; tb += 2) {
                const uint32_t dt = tmem + (uint32_t)((sa + tb) * 64);
                const uint64_t ad = a0 + (uint64_t)((sa * 2 * kTileBytes) >> 4);
                const uint64_t bd = b0 + (uint64_t)((tb * kTileBytes) >> 4);
                const uint32_t id = tb + 1 < S - sa ? idesc2 : idesc;
                mma_f16(dt, ad, bd, (sa == 0 && first) ? 0u : 1u, id);
                mma_f16(dt, ad + (256 >> 4), bd + (256 >> 4), 1u, id);
              }
          }
          mma_commit(smem_u32(&bar_free[stg]));
          if (last) {
            mma_commit(smem_u32(&bar_acc_full));
            q++;
          }
        }
      }
      if (!ok) {
        abort_flag = 1;
        // the MMAs already issued complete in order: wait (bounded) for the
        // last commit before the accumulators are freed
        if (g > 0) mbar_wait(smem_u32(&bar_free[(g - 1) % kOzStages]), ((g - 1) / kOzStages) & 1);
      }
    }
  } else {
    // ---- drain and epilogue (warps 0-7) ----
    const int quarter = warp & 3, hcol = warp >> 2;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(hcol * 32);
    // 64-bit totals after the accumulators: value j of the half at 2j (lo), 2j + 1 (hi)
    const uint32_t ttot = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(S * 64 + hcol * 64);
    // ATMEM: the totals in shared memory after the ring, output j of lane l
    // of warp w at [(w * 32 + j) * 32 + l] (lanes contiguous)
    long long* stot = reinterpret_cast<long long*>(smem + kOzStages * kStage) + warp * 32 * 32 + lane;
    uint32_t q = 0;
    for (int t = blockIdx.x; t < ntasks && ok; t += gridDim.x) {
      const OzTask task = tasks[t];
      const OzDesc* dp = descs + task.d;
      int kb0, nkb;
      task_range(*dp, task.ks, kb0, nkb);
      if (nkb <= 0) continue;
      // the fields the epilogue needs, as scalars (kept in registers)
      const int dM = dp->M, dN = dp->N, ldc = dp->ldc, cscale = dp->cscale, coff = dp->coff;
      const int atomic = dp->atomic;
      const int* __restrict__ eB = dp->eB;
      double* __restrict__ Cp = dp->C;
      const bool neg = dp->alpha < 0.0;  // alpha is +-1: its sign goes into the doubles
      const int nchunks = (nkb + kChunk - 1) / kChunk;
      const int r = task.tm * 128 + quarter * 32 + lane;
      const int nb = task.tn * 64 + hcol * 32;
      const int ea_row = r < dM ? dp->eA[r] : 0;
      for (int c = 0; c < nchunks; c++, q++) {
        if (!mbar_wait(smem_u32(&bar_acc_full), q & 1) || abort_flag) {
          ok = false;
          break;
        }
        fence_after();
        // the chunk's S accumulators -> one 64-bit partial sum per output,
        // added into the running totals in tensor memory, in two rounds of
        // 16 outputs (32 TMEM columns of totals) each
#pragma unroll 1
        for (int g2 = 0; g2 < 2; g2++) {
          long long part[16];
#pragma unroll
          for (int j = 0; j < 16; j++) part[j] = 0;
#pragma unroll 1
          for (int dd = 0; dd < S; dd++) {
            const int shift = 7 * (S - 1 - dd);
            uint32_t v[16];
            tmem_ld16(trow + (uint32_t)(dd * 64 + g2 * 16), v);
#pragma unroll
            for (int j = 0; j < 16; j++)
              part[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << shift;
          }
          if (g2 == 1) {
            // every accumulator read: the MMAs of the next chunk may start
            // while the totals (other columns) are updated
            fence_before();
            __syncwarp();
            if (lane == 0)
              asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar_acc_empty))
                           : "memory");
          }
          if (ATMEM) {
#pragma unroll
            for (int j = 0; j < 16; j++) {
              long long* tp = stot + (g2 * 16 + j) * 32;
              *tp = c > 0 ? *tp + part[j] : part[j];
            }
          } else {
            uint32_t tv[32];
            if (c > 0) tmem_ld32(ttot + (uint32_t)(g2 * 32), tv);
#pragma unroll
            for (int j = 0; j < 16; j++) {
              long long tt = part[j];
              if (c > 0) tt += (long long)(((unsigned long long)tv[2 * j + 1] << 32) | tv[2 * j]);
              tv[2 * j] = (uint32_t)tt;
              tv[2 * j + 1] = (uint32_t)((unsigned long long)tt >> 32);
            }
            tmem_st32(ttot + (uint32_t)(g2 * 32), tv);
          }
        }
        // the totals are written before the epilogue reads them (same warp)
        fence_before();
        __syncwarp();
        // (warp-uniform: the tensor-memory loads below need the whole warp)
        if (c != nchunks - 1) continue;
        // last chunk: the totals become the FP64 outputs (while the MMAs of
        // the next task already run)
        const int ea = ea_row - 14 - 7 * (S - 1);
#pragma unroll 1
        for (int g2 = 0; g2 < 2; g2++) {
          uint32_t tv[32];
          if (!ATMEM) tmem_ld32(ttot + (uint32_t)(g2 * 32), tv);
          if (r < dM) {
#pragma unroll
            for (int j = 0; j < 16; j++) {
              const int n = nb + g2 * 16 + j;
              if (n < dN) {
                const long long tt =
                    ATMEM ? stot[(g2 * 16 + j) * 32]
                          : (long long)(((unsigned long long)tv[2 * j + 1] << 32) | tv[2 * j]);
                const double v = scaled_int_to_double(tt, ea + eB[n], neg);
                double* cp = Cp + (r + (int64_t)n * ldc) * cscale + coff;
                if (atomic) atomicAdd(cp, v); else *cp = v;
              }
            }
          }
          __syncwarp();  // converged again for the next tensor-memory load
        }
      }
    }
    if (!ok) abort_flag = 1;
  }
  if (!ok && lane == 0) atomicExch(err, DEV_TIMEOUT);
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

template <int S, bool ATMEM>
constexpr int gemm_smem() {
  return oz_stages<S, ATMEM>() * S * 3 * kTileBytes + (ATMEM ? kOzDrainWarps * 32 * 32 * 8 : 0);
}

// Failure-path check: wait on an mbarrier that nothing will complete, with a
// short budget, and record the timeout like any other bounded wait.
__global__ void wait_selftest_kernel(int* err, unsigned long long budget_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0, budget_ns)) set_error(err, DEV_TIMEOUT, 0);
}

__global__ void zero_kernel(const CopySeg* __restrict__ segs, int nseg) {
  for (int s = blockIdx.y; s < nseg; s += gridDim.y) {
    const CopySeg g = segs[s];
    double* b = (double*)g.dst;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.count;
         e += (int64_t)gridDim.x * blockDim.x)
      b[e] = 0.0;
  }
}

}  // namespace

cudaError_t prepare_ozaki_kernels() {
  cudaError_t e;
  e = cudaFuncSetAttribute(gslice_kernel<cdouble, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)gslice_smem<cdouble>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(gslice_kernel<cdouble, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)gslice_smem<cdouble>());
  if (e != cudaSuccess) return e;
#define PSELINV_OZ_ATTR(S, AT)                                                               \
  e = cudaFuncSetAttribute(ozaki_gemm_kernel<S, AT>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           gemm_smem<S, AT>());                                                 \
  if (e != cudaSuccess) return e;
  PSELINV_OZ_ATTR(4, false)
  PSELINV_OZ_ATTR(5, false)
  PSELINV_OZ_ATTR(6, false)
  PSELINV_OZ_ATTR(4, true)
  PSELINV_OZ_ATTR(5, true)
  PSELINV_OZ_ATTR(6, true)
#undef PSELINV_OZ_ATTR
  return cudaSuccess;
}

void launch_slice(const SliceDesc* descs, const SliceTask* tasks, int ntasks, bool maxima,
                  cudaStream_t st) {
  if (ntasks <= 0) return;
  const int grid = ntasks < 152 * 16 ? ntasks : 152 * 16;
  if (maxima)
    slice_max_kernel<<<grid, kSliceThreads, 0, st>>>(descs, tasks, ntasks);
  else
    slice_kernel<<<grid, kSliceThreads, 0, st>>>(descs, tasks, ntasks);
}

namespace {
// Row and column maxima of one chunk of up to 128 rows of a stored block
// of Ainv (see MaxTask): warp w takes the columns w, w + 8, ..., a lane the
// rows lane + 32 i of each (coalesced down the column-major block); a
// column's maximum is a warp reduction, a row's a reduction over the warps
// in shared memory; one atomicMax per row and per column of the chunk.
constexpr int kMaxRows = kOutMaxRows;
template <typename T>
__global__ void __launch_bounds__(kSliceThreads)
out_maxima_kernel(SymDev S, const T* __restrict__ store, const MaxTask* __restrict__ tasks,
                  int ntasks, unsigned long long* rcmax) {
  constexpr int kWarps = kSliceThreads / 32;
  __shared__ unsigned long long rowm[kWarps][kMaxRows];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const MaxTask task = tasks[t];
    const int K = task.K, s = S.sn_width[K], f = S.sn_first[K];
    const int r0 = task.rc * kMaxRows, nr = min(kMaxRows, task.nrows - r0);
    const T* blk = store + (int64_t)task.inst * S.storage + task.off + r0;
    unsigned long long* rmax = rcmax + (int64_t)task.inst * 2 * S.n;
    unsigned long long* cmax = rmax + S.n;
    // where the block's rows and columns lie among the rows / columns of Ainv
    unsigned long long* rdst = task.which == 2 ? cmax : rmax;
    unsigned long long* cdst = task.which == 2 ? rmax : cmax;
    unsigned long long m[kMaxRows / 32];
#pragma unroll
    for (int i = 0; i < kMaxRows / 32; i++) m[i] = 0;
    for (int tc = warp; tc < s; tc += kWarps) {
      const T* col = blk + (int64_t)tc * task.nrows;
      unsigned long long cm = 0;
#pragma unroll
      for (int i = 0; i < kMaxRows / 32; i++) {
        const int r = lane + 32 * i;
        const unsigned long long v = r < nr ? abs_bits_max(col[r]) : 0ull;
        m[i] = max(m[i], v);
        cm = max(cm, v);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cm = max(cm, __shfl_xor_sync(0xffffffffu, cm, o));
      if (lane == 0 && cm) atomicMax(cdst + f + tc, cm);
    }
#pragma unroll
    for (int i = 0; i < kMaxRows / 32; i++) rowm[warp][lane + 32 * i] = m[i];
    __syncthreads();
    if (tid < nr) {
      unsigned long long x = 0;
#pragma unroll
      for (int w = 0; w < kWarps; w++) x = max(x, rowm[w][tid]);
      const int32_t* R = task.which == 0 ? nullptr
                         : task.upanel   ? S.urows + S.urows_ptr[K]
                                         : S.lrows + S.rows_ptr[K];
      if (x) atomicMax(rdst + (task.which == 0 ? f + r0 + tid : R[r0 + tid]), x);
    }
    __syncthreads();
  }
}
}  // namespace

void launch_out_maxima(int dtype, const SymDev& S, const void* store, const MaxTask* tasks,
                       int ntasks, unsigned long long* rcmax, cudaStream_t st) {
  if (ntasks <= 0) return;
  const int grid = ntasks < 152 * 8 ? ntasks : 152 * 8;
  if (dtype == DT_F64)
    out_maxima_kernel<double><<<grid, kSliceThreads, 0, st>>>(S, (const double*)store, tasks,
                                                              ntasks, rcmax);
  else
    out_maxima_kernel<cdouble><<<grid, kSliceThreads, 0, st>>>(S, (const cdouble*)store, tasks,
                                                               ntasks, rcmax);
}

void launch_gslice(int dtype, const SymDev& S, const void* store, const SliceDesc* descs,
                   const GTileTask* gtasks, int ngt, const SliceTask* stasks, int nst, bool maxima,
                   unsigned long long* rcmax, cudaStream_t st) {
  const int ntasks = ngt + nst;
  if (ntasks <= 0) return;
  const int grid = ntasks < 152 * 8 ? ntasks : 152 * 8;
  if (dtype == DT_F64) {
    const size_t sm = gslice_smem<double>();
    if (maxima)
      gslice_kernel<double, true><<<grid, kSliceThreads, sm, st>>>(
          S, (const double*)store, descs, gtasks, ngt, stasks, nst, rcmax);
    else
      gslice_kernel<double, false><<<grid, kSliceThreads, sm, st>>>(
          S, (const double*)store, descs, gtasks, ngt, stasks, nst, rcmax);
  } else {
    const size_t sm = gslice_smem<cdouble>();
    if (maxima)
      gslice_kernel<cdouble, true><<<grid, kSliceThreads, sm, st>>>(
          S, (const cdouble*)store, descs, gtasks, ngt, stasks, nst, rcmax);
    else
      gslice_kernel<cdouble, false><<<grid, kSliceThreads, sm, st>>>(
          S, (const cdouble*)store, descs, gtasks, ngt, stasks, nst, rcmax);
  }
}

void launch_ozaki_gemm(int S, const OzDesc* descs, const OzTask* tasks, int ntasks, int* err,
                       bool persistent, bool a_tmem, cudaStream_t st) {
  if (ntasks <= 0) return;
  // one CTA fits an SM (shared memory and tensor memory): a persistent grid
  // on the sweep's stream; one task per CTA on the normalisation stream, so
  // that its CTAs leave SMs to the sweep between tasks
  const int grid = persistent && ntasks > 152 ? 152 : ntasks;
#define PSELINV_OZ_LAUNCH(SS, AT)                                                        \
  ozaki_gemm_kernel<SS, AT><<<grid, kOzThreads, gemm_smem<SS, AT>(), st>>>(descs, tasks, \
                                                                          ntasks, err)
  if (a_tmem) {
    switch (S) {
      case 4: PSELINV_OZ_LAUNCH(4, true); break;
      case 5: PSELINV_OZ_LAUNCH(5, true); break;
      default: PSELINV_OZ_LAUNCH(6, true); break;
    }
  } else {
    switch (S) {
      case 4: PSELINV_OZ_LAUNCH(4, false); break;
      case 5: PSELINV_OZ_LAUNCH(5, false); break;
      default: PSELINV_OZ_LAUNCH(6, false); break;
    }
  }
#undef PSELINV_OZ_LAUNCH
}

void launch_wait_selftest(int* err, unsigned long long budget_ns, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(err, budget_ns);
}

void launch_zero(const CopySeg* segs, int nseg, int per_seg, cudaStream_t st) {
  if (nseg <= 0) return;
  dim3 grid(per_seg > 0 ? per_seg : 8, nseg < 65535 ? nseg : 65535);
  zero_kernel<<<grid, 256, 0, st>>>(segs, nseg);
}

}  // namespace pselinv
