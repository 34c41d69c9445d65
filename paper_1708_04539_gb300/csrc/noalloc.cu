// Allocation-free entry point: inverse of one LU-factored diagonal block.
//
// Some callers cannot allocate device memory at all: code that runs while a
// framework's caching allocator owns the whole device, plug-ins handed a
// fixed memory budget, or host code that must not call cudaMalloc /
// cudaFree because those calls synchronise the device.  For them this file
// offers pselinv_block_inverse_noalloc(), a variant of the handle-based
// normalisation (triangular inverses into scratch, then one product) whose
// scratch lives in a fixed-size array compiled into the library instead of
// a handle's arena.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (2 MiB) until the process exits.  Its host-side name is
// only a stand-in, so the per-device address is looked up once with
// cudaGetSymbolAddress, on the first call made on that device, with the
// device current, and kept for the life of the process (so the entry point
// must not be used on a device after cudaDeviceReset of that device: the
// module, and with it the array, may then live at another address).  All
// calls share the array and it keeps the last call's contents; calls that
// overlap on the GPU (different streams, or the same device from several
// threads) race on it and must be serialised by the caller.  Both pointers
// must be device memory of the current device (checked with
// cudaPointerGetAttributes; anything else is refused before any launch).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "device.cuh"
#include "pselinv.h"

namespace pselinv {
namespace {

constexpr int kMaxS = PSELINV_NOALLOC_MAX_S;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// 2 * 256 * 256 complex128 scalars = 2 MiB: (L_KK)^{-1} and (U_KK)^{-1}
__device__ __align__(256) unsigned char g_noalloc_scratch[2ull * kMaxS * kMaxS * 16];

std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Triangular inverses of the s x s block (column-major, leading dimension
// ld): blocks [0, nchunk) give (L)^{-1} (unit lower), [nchunk, 2 nchunk)
// give (U)^{-1}; each warp solves one column into W (s x s, ld = s).
template <typename T>
__global__ void __launch_bounds__(kThreads)
block_tri_inv_kernel(const T* __restrict__ blk, int ld, int s, T* W) {
  extern __shared__ unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunk = (s + 7) / 8;
  const int which = blockIdx.x / nchunk;
  const int j = (blockIdx.x % nchunk) * 8 + warp;
  if (j >= s) return;
  T* x = reinterpret_cast<T*>(smem_raw) + (int64_t)warp * s;
  T* out = W + (int64_t)which * s * s;
  for (int i = lane; i < s; i += 32) x[i] = (i == j) ? sc_one(T()) : sc_zero(T());
  __syncwarp();
  if (which == 0) {
    for (int k = j; k < s - 1; k++) {
      const T xk = x[k];
      __syncwarp();
      if (!is_zero(xk))
        for (int i = k + 1 + lane; i < s; i += 32)
          x[i] = sub_s(x[i], mul_s(blk[i + (int64_t)k * ld], xk));
      __syncwarp();
    }
  } else {
    for (int k = j; k >= 0; k--) {
      const T xk = div_s(x[k], blk[k + (int64_t)k * ld]);
      __syncwarp();
      if (lane == 0) x[k] = xk;
      for (int i = lane; i < k; i += 32) x[i] = sub_s(x[i], mul_s(blk[i + (int64_t)k * ld], xk));
      __syncwarp();
    }
  }
  for (int i = lane; i < s; i += 32) out[i + (int64_t)j * s] = x[i];
}

// out = Uinv * Linv, one BM x BN tile per CTA (W holds Linv then Uinv).
template <typename T, int BM, int BN, int BK>
__global__ void __launch_bounds__(kThreads)
block_product_kernel(const T* __restrict__ W, int s, T* out, int ldo) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ T sa[BK][BM];
  __shared__ T sb[BK][BN];
  const T* Linv = W;
  const T* Uinv = W + (int64_t)s * s;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; i++)
#pragma unroll
    for (int j = 0; j < TN; j++) acc[i][j] = sc_zero(T());
  for (int k0 = 0; k0 < s; k0 += BK) {
    for (int e = tid; e < BM * BK; e += kThreads) {
      const int mm = e % BM, kk = e / BM, m = m0 + mm, k = k0 + kk;
      sa[kk][mm] = (m < s && k < s) ? Uinv[m + (int64_t)k * s] : sc_zero(T());
    }
    for (int e = tid; e < BK * BN; e += kThreads) {
      const int kk = e % BK, nn = e / BK, n = n0 + nn, k = k0 + kk;
      sb[kk][nn] = (n < s && k < s) ? Linv[k + (int64_t)n * s] : sc_zero(T());
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk++) {
#pragma unroll
      for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++)
          acc[i][j] = fma_s(sa[kk][tx + 16 * i], sb[kk][ty + 16 * j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; i++)
#pragma unroll
    for (int j = 0; j < TN; j++) {
      const int m = m0 + tx + 16 * i, n = n0 + ty + 16 * j;
      if (m < s && n < s) out[m + (int64_t)n * ldo] = acc[i][j];
    }
}

template <typename T, int BM, int BN>
cudaError_t run(const void* lu, int ld_in, int s, void* inv, int ld_out, cudaStream_t st) {
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return e;
  T* W = static_cast<T*>(scratch);
  const int nchunk = (s + 7) / 8;
  const size_t smem = (size_t)(kThreads / 32) * s * sizeof(T);
  block_tri_inv_kernel<T><<<2 * nchunk, kThreads, smem, st>>>(static_cast<const T*>(lu), ld_in, s,
                                                             W);
  dim3 grid((s + BM - 1) / BM, (s + BN - 1) / BN);
  block_product_kernel<T, BM, BN, 16><<<grid, kThreads, 0, st>>>(W, s, static_cast<T*>(inv),
                                                                 ld_out);
  return cudaGetLastError();
}

// Whether p is device (or managed) memory of the current device: a host
// pointer, or one of another device, would make the kernels fault.
bool on_current_device(const void* p) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace
}  // namespace pselinv

extern "C" int pselinv_block_inverse_noalloc(int dtype, int64_t s, const void* lu_block,
                                             int64_t ld_in, void* inv_out, int64_t ld_out,
                                             void* stream) {
  using namespace pselinv;
  if (dtype != PSELINV_F64 && dtype != PSELINV_C128) return PSELINV_ERR_ARG;
  if (s < 1 || s > PSELINV_NOALLOC_MAX_S || ld_in < s || ld_out < s || !lu_block || !inv_out)
    return PSELINV_ERR_ARG;
  if (!on_current_device(lu_block) || !on_current_device(inv_out)) return PSELINV_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const cudaError_t e =
      dtype == PSELINV_F64
          ? run<double, 64, 64>(lu_block, (int)ld_in, (int)s, inv_out, (int)ld_out, st)
          : run<cdouble, 32, 32>(lu_block, (int)ld_in, (int)s, inv_out, (int)ld_out, st);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return PSELINV_ERR_CUDA;
  }
  return PSELINV_OK;
}
