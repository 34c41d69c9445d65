// Learned cost model of the launch shapes (not from the paper): a small MLP
//   x (16) -> tanh(W1 x + b1) (H) -> tanh(W2 h1 + b2) (H) -> w3 . h2 + b3
// predicting log(milliseconds) of one launch from the shape features of the
// step and the candidate launch parameter.  It is trained on the autotuner's
// own measurements by a hand-written single-CTA kernel that runs every epoch
// of full-batch Adam (forward, backward, update) in one launch, and queried
// by a batched inference kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "pselinv.h"

namespace {

constexpr int kIn = 16;
constexpr int kMaxHidden = 64;
constexpr int kTrainThreads = 1024;

struct Layout {
  int H;
  int w1, b1, w2, b2, w3, b3, total;
  explicit Layout(int h) : H(h) {
    w1 = 0;
    b1 = w1 + h * kIn;
    w2 = b1 + h;
    b2 = w2 + h * h;
    w3 = b2 + h;
    b3 = w3 + h;
    total = b3 + 1;
  }
};

// input encoding of one record (see pselinv_model_* in the header)
void encode(const pselinv_tune_record& r, float* x) {
  for (int i = 0; i < 8; i++) x[i] = r.feat[i] / 32.0f;
  const bool gemm = r.kind == PSELINV_STEP_GEMM;
  x[8] = gemm ? 1.0f : 0.0f;
  x[9] = gemm ? 0.0f : 1.0f;
  x[10] = (gemm && r.param == 0) ? 1.0f : 0.0f;
  x[11] = (gemm && r.param == 1) ? 1.0f : 0.0f;
  x[12] = (gemm && r.param == 2) ? 1.0f : 0.0f;
  x[13] = gemm ? 0.0f : std::log2((float)(r.param > 0 ? r.param : 1)) / 4.0f;
  x[14] = r.slot / 2.0f;
  x[15] = (float)r.precision;
}

// SplitMix64 (Steele, Lea, Flood 2014) for the initial weights
uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ void forward_one(const float* P, const Layout& L, const float* x, float* h1,
                                            float* h2, float* out) {
  for (int j = 0; j < L.H; j++) {
    float a = P[L.b1 + j];
    for (int k = 0; k < kIn; k++) a = fmaf(P[L.w1 + j * kIn + k], x[k], a);
    h1[j] = tanhf(a);
  }
  for (int j = 0; j < L.H; j++) {
    float a = P[L.b2 + j];
    for (int k = 0; k < L.H; k++) a = fmaf(P[L.w2 + j * L.H + k], h1[k], a);
    h2[j] = tanhf(a);
  }
  float o = P[L.b3];
  for (int k = 0; k < L.H; k++) o = fmaf(P[L.w3 + k], h2[k], o);
  *out = o;
}

// One CTA: `epochs` full-batch Adam steps on the mean squared error of
// log-time (epochs = 0: gradient and loss only, parameters untouched).
// H1, H2, D1, D2: n x H scratch (activations and their back-propagated errors).
__global__ void __launch_bounds__(kTrainThreads)
mlp_train_kernel(Layout L, const float* __restrict__ X, const float* __restrict__ y, int n,
                 int epochs, float lr, float* params, float* madam, float* vadam, float* grad,
                 float* H1, float* H2, float* D1, float* D2, float* D3, float* loss_out) {
  extern __shared__ float sP[];  // parameters
  __shared__ float red[kTrainThreads / 32];
  const int tid = threadIdx.x;
  for (int i = tid; i < L.total; i += blockDim.x) sP[i] = params[i];
  __syncthreads();
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int iters = epochs > 0 ? epochs : 1;
  for (int ep = 0; ep < iters; ep++) {
    // forward + output error
    float lsum = 0.0f;
    for (int i = tid; i < n; i += blockDim.x) {
      float out;
      forward_one(sP, L, X + (int64_t)i * kIn, H1 + (int64_t)i * L.H, H2 + (int64_t)i * L.H, &out);
      const float e = out - y[i];
      D3[i] = 2.0f * e / n;
      lsum += e * e;
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((tid & 31) == 0) red[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
      float t = 0.0f;
      for (int w = 0; w < (int)(blockDim.x / 32); w++) t += red[w];
      *loss_out = t / n;
    }
    // back-propagate to the hidden layers
    for (int i = tid; i < n; i += blockDim.x) {
      const float* h1 = H1 + (int64_t)i * L.H;
      const float* h2 = H2 + (int64_t)i * L.H;
      float* d2 = D2 + (int64_t)i * L.H;
      float* d1 = D1 + (int64_t)i * L.H;
      const float d3 = D3[i];
      for (int j = 0; j < L.H; j++) d2[j] = sP[L.w3 + j] * d3 * (1.0f - h2[j] * h2[j]);
      for (int k = 0; k < L.H; k++) {
        float a = 0.0f;
        for (int j = 0; j < L.H; j++) a = fmaf(sP[L.w2 + j * L.H + k], d2[j], a);
        d1[k] = a * (1.0f - h1[k] * h1[k]);
      }
    }
    __syncthreads();
    // parameter gradients: one thread per parameter, sum over samples
    for (int p = tid; p < L.total; p += blockDim.x) {
      float g = 0.0f;
      if (p < L.b1) {
        const int j = p / kIn, k = p % kIn;
        for (int i = 0; i < n; i++) g = fmaf(D1[(int64_t)i * L.H + j], X[(int64_t)i * kIn + k], g);
      } else if (p < L.w2) {
        const int j = p - L.b1;
        for (int i = 0; i < n; i++) g += D1[(int64_t)i * L.H + j];
      } else if (p < L.b2) {
        const int j = (p - L.w2) / L.H, k = (p - L.w2) % L.H;
        for (int i = 0; i < n; i++) g = fmaf(D2[(int64_t)i * L.H + j], H1[(int64_t)i * L.H + k], g);
      } else if (p < L.w3) {
        const int j = p - L.b2;
        for (int i = 0; i < n; i++) g += D2[(int64_t)i * L.H + j];
      } else if (p < L.b3) {
        const int k = p - L.w3;
        for (int i = 0; i < n; i++) g = fmaf(D3[i], H2[(int64_t)i * L.H + k], g);
      } else {
        for (int i = 0; i < n; i++) g += D3[i];
      }
      grad[p] = g;
    }
    __syncthreads();
    if (epochs > 0) {
      const float c1 = 1.0f - powf(b1, (float)(ep + 1)), c2 = 1.0f - powf(b2, (float)(ep + 1));
      for (int p = tid; p < L.total; p += blockDim.x) {
        const float g = grad[p];
        const float m = b1 * madam[p] + (1.0f - b1) * g;
        const float v = b2 * vadam[p] + (1.0f - b2) * g * g;
        madam[p] = m;
        vadam[p] = v;
        sP[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < L.total; i += blockDim.x) params[i] = sP[i];
}

__global__ void mlp_predict_kernel(Layout L, const float* __restrict__ params,
                                   const float* __restrict__ X, int n, float* out) {
  float h1[kMaxHidden], h2[kMaxHidden];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float o;
  forward_one(params, L, X + (int64_t)i * kIn, h1, h2, &o);
  out[i] = o;
}

}  // namespace

struct pselinv_model {
  Layout L{32};
  int device = 0;
  float* params = nullptr;  // device
  float* madam = nullptr;
  float* vadam = nullptr;
  float* grad = nullptr;
  float* loss = nullptr;
  int64_t cap = 0;          // samples the scratch holds
  float* scratch = nullptr; // X | y | H1 | H2 | D1 | D2 | D3 | out
  float y_mean = 0.0f;
};

namespace {

int ensure_scratch(pselinv_model* m, int64_t n) {
  if (n <= m->cap) return PSELINV_OK;
  cudaFree(m->scratch);
  m->scratch = nullptr;
  const size_t floats = (size_t)n * (kIn + 1 + 4 * m->L.H + 2) + 64;
  if (cudaMalloc(&m->scratch, floats * sizeof(float)) != cudaSuccess) {
    (void)cudaGetLastError();
    m->cap = 0;
    return PSELINV_ERR_OOM;
  }
  m->cap = n;
  return PSELINV_OK;
}

struct Views {
  float *X, *y, *H1, *H2, *D1, *D2, *D3, *out;
};
Views views(pselinv_model* m, int64_t n) {
  Views v;
  v.X = m->scratch;
  v.y = v.X + n * kIn;
  v.H1 = v.y + n;
  v.H2 = v.H1 + n * m->L.H;
  v.D1 = v.H2 + n * m->L.H;
  v.D2 = v.D1 + n * m->L.H;
  v.D3 = v.D2 + n * m->L.H;
  v.out = v.D3 + n;
  return v;
}

int upload_records(pselinv_model* m, const pselinv_tune_record* recs, int64_t n, bool targets,
                   cudaStream_t st) {
  std::vector<float> hx((size_t)n * kIn), hy(targets ? (size_t)n : 0);
  for (int64_t i = 0; i < n; i++) {
    encode(recs[i], hx.data() + i * kIn);
    if (targets) hy[i] = (float)std::log(recs[i].ms > 1e-6 ? recs[i].ms : 1e-6);
  }
  const Views v = views(m, n);
  if (cudaMemcpyAsync(v.X, hx.data(), hx.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PSELINV_ERR_CUDA;
  if (targets &&
      cudaMemcpyAsync(v.y, hy.data(), hy.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PSELINV_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? PSELINV_OK : PSELINV_ERR_CUDA;
}

int run_train(pselinv_model* m, int64_t n, int epochs, float lr, cudaStream_t st) {
  const Views v = views(m, n);
  const size_t smem = (size_t)m->L.total * sizeof(float);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
    return PSELINV_ERR_CUDA;
  mlp_train_kernel<<<1, kTrainThreads, smem, st>>>(m->L, v.X, v.y, (int)n, epochs, lr, m->params,
                                                  m->madam, m->vadam, m->grad, v.H1, v.H2, v.D1,
                                                  v.D2, v.D3, m->loss);
  if (cudaGetLastError() != cudaSuccess) return PSELINV_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? PSELINV_OK : PSELINV_ERR_CUDA;
}

}  // namespace

extern "C" {

int pselinv_model_create(int32_t hidden, uint64_t seed, pselinv_model_t* out) {
  if (!out || hidden < 1 || hidden > kMaxHidden) return PSELINV_ERR_ARG;
  *out = nullptr;
  pselinv_model* m = new (std::nothrow) pselinv_model();
  if (!m) return PSELINV_ERR_OOM;
  m->L = Layout(hidden);
  cudaGetDevice(&m->device);
  const size_t bytes = (size_t)m->L.total * sizeof(float);
  if (cudaMalloc(&m->params, bytes) != cudaSuccess || cudaMalloc(&m->madam, bytes) != cudaSuccess ||
      cudaMalloc(&m->vadam, bytes) != cudaSuccess || cudaMalloc(&m->grad, bytes) != cudaSuccess ||
      cudaMalloc(&m->loss, sizeof(float)) != cudaSuccess) {
    (void)cudaGetLastError();
    pselinv_model_free(m);
    return PSELINV_ERR_OOM;
  }
  // Glorot-style uniform weights, zero biases
  std::vector<float> p(m->L.total, 0.0f);
  uint64_t st = seed;
  auto uni = [&](float a) {
    const double u = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
    return (float)((2.0 * u - 1.0) * a);
  };
  const float a1 = std::sqrt(6.0f / (kIn + hidden)), a2 = std::sqrt(6.0f / (2 * hidden)),
              a3 = std::sqrt(6.0f / (hidden + 1));
  for (int i = 0; i < hidden * kIn; i++) p[m->L.w1 + i] = uni(a1);
  for (int i = 0; i < hidden * hidden; i++) p[m->L.w2 + i] = uni(a2);
  for (int i = 0; i < hidden; i++) p[m->L.w3 + i] = uni(a3);
  if (cudaMemcpy(m->params, p.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->madam, 0, bytes) != cudaSuccess || cudaMemset(m->vadam, 0, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    pselinv_model_free(m);
    return PSELINV_ERR_CUDA;
  }
  *out = m;
  return PSELINV_OK;
}

int pselinv_model_train(pselinv_model_t m, const pselinv_tune_record* recs, int64_t n, int32_t epochs,
                        float lr, void* stream, float* final_loss) {
  if (!m || !recs || n < 1 || epochs < 1 || !(lr > 0.0f)) return PSELINV_ERR_ARG;
  cudaSetDevice(m->device);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_scratch(m, n);
  if (rc != PSELINV_OK) return rc;
  rc = upload_records(m, recs, n, true, st);
  if (rc != PSELINV_OK) return rc;
  rc = run_train(m, n, epochs, lr, st);
  if (rc != PSELINV_OK) return rc;
  if (final_loss && cudaMemcpy(final_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PSELINV_ERR_CUDA;
  return PSELINV_OK;
}

int pselinv_model_gradients(pselinv_model_t m, const pselinv_tune_record* recs, int64_t n,
                            float* grad_out, float* loss_out, void* stream) {
  if (!m || !recs || n < 1 || !grad_out) return PSELINV_ERR_ARG;
  cudaSetDevice(m->device);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_scratch(m, n);
  if (rc != PSELINV_OK) return rc;
  rc = upload_records(m, recs, n, true, st);
  if (rc != PSELINV_OK) return rc;
  rc = run_train(m, n, 0, 1.0f, st);
  if (rc != PSELINV_OK) return rc;
  if (cudaMemcpy(grad_out, m->grad, (size_t)m->L.total * sizeof(float), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return PSELINV_ERR_CUDA;
  if (loss_out && cudaMemcpy(loss_out, m->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PSELINV_ERR_CUDA;
  return PSELINV_OK;
}

int pselinv_model_predict(pselinv_model_t m, const pselinv_tune_record* recs, int64_t n,
                          double* pred_ms, void* stream) {
  if (!m || !recs || n < 1 || !pred_ms) return PSELINV_ERR_ARG;
  cudaSetDevice(m->device);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_scratch(m, n);
  if (rc != PSELINV_OK) return rc;
  rc = upload_records(m, recs, n, false, st);
  if (rc != PSELINV_OK) return rc;
  const Views v = views(m, n);
  mlp_predict_kernel<<<(int)((n + 127) / 128), 128, 0, st>>>(m->L, m->params, v.X, (int)n, v.out);
  if (cudaGetLastError() != cudaSuccess) return PSELINV_ERR_CUDA;
  std::vector<float> o((size_t)n);
  if (cudaMemcpyAsync(o.data(), v.out, (size_t)n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PSELINV_ERR_CUDA;
  for (int64_t i = 0; i < n; i++) pred_ms[i] = std::exp((double)o[i]);
  return PSELINV_OK;
}

int pselinv_model_get_params(pselinv_model_t m, float* out, int64_t cap, int64_t* count) {
  if (!m || !count) return PSELINV_ERR_ARG;
  *count = m->L.total;
  if (out && cap >= m->L.total) {
    cudaSetDevice(m->device);
    if (cudaMemcpy(out, m->params, (size_t)m->L.total * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return PSELINV_ERR_CUDA;
  }
  return PSELINV_OK;
}

int pselinv_model_set_params(pselinv_model_t m, const float* in, int64_t count) {
  if (!m || !in || count != m->L.total) return PSELINV_ERR_ARG;
  cudaSetDevice(m->device);
  const size_t bytes = (size_t)m->L.total * 4;
  if (cudaMemcpy(m->params, in, bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->madam, 0, bytes) != cudaSuccess || cudaMemset(m->vadam, 0, bytes) != cudaSuccess)
    return PSELINV_ERR_CUDA;
  return PSELINV_OK;
}

int pselinv_model_encode(const pselinv_tune_record* recs, int64_t n, float* x_out) {
  if (!recs || !x_out || n < 0) return PSELINV_ERR_ARG;
  for (int64_t i = 0; i < n; i++) encode(recs[i], x_out + i * kIn);
  return PSELINV_OK;
}

void pselinv_model_free(pselinv_model_t m) {
  if (!m) return;
  cudaSetDevice(m->device);
  cudaFree(m->params);
  cudaFree(m->madam);
  cudaFree(m->vadam);
  cudaFree(m->grad);
  cudaFree(m->loss);
  cudaFree(m->scratch);
  delete m;
}

}  // extern "C"
