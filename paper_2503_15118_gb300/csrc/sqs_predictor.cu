// Learned capacity predictor: a small MLP that predicts, from structural
// features of an interference step, log2 of the ratio between the branch
// count after the step (merged and pruned) and before it.  The runtime sizes
// the merge from the prediction instead of the worst-case bound; an
// overflow is detected on the device and the step re-run at the exact size.
//
// Network: F inputs -> H tanh -> H tanh -> 1 linear, FP32, weights in one
// device buffer.  Forward, backward (mean-squared error) and Adam are
// hand-written kernels; one CTA handles a tile of samples, one thread one
// sample, weights read from shared memory, gradients reduced through
// shared-memory atomics then one global atomic per weight per CTA.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/sqs.h"
#include "sqs_internal.h"

namespace sqs {

constexpr int F = SQS_PRED_FEATURES;
constexpr int H = SQS_PRED_HIDDEN;
// Parameter layout: W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.
constexpr int kW1 = 0, kB1 = kW1 + H * F, kW2 = kB1 + H, kB2 = kW2 + H * H, kW3 = kB2 + H,
              kB3 = kW3 + H, kNP = kB3 + 1;
static_assert(kNP == SQS_PRED_PARAMS, "parameter count");

constexpr int kMlpThreads = 128;

__device__ __forceinline__ void mlp_forward_one(const float* p, const float* x, float* a1,
                                                float* a2, float& y) {
  for (int h = 0; h < H; ++h) {
    float s = p[kB1 + h];
    for (int f = 0; f < F; ++f) s = fmaf(p[kW1 + h * F + f], x[f], s);
    a1[h] = tanhf(s);
  }
  for (int h = 0; h < H; ++h) {
    float s = p[kB2 + h];
    for (int k = 0; k < H; ++k) s = fmaf(p[kW2 + h * H + k], a1[k], s);
    a2[h] = tanhf(s);
  }
  float s = p[kB3];
  for (int h = 0; h < H; ++h) s = fmaf(p[kW3 + h], a2[h], s);
  y = s;
}

__global__ void __launch_bounds__(kMlpThreads)
    k_mlp_forward(const float* params, const float* X, int n, float* Y) {
  __shared__ float p[kNP];
  for (int i = threadIdx.x; i < kNP; i += blockDim.x) p[i] = params[i];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[F], a1[H], a2[H], y;
  for (int f = 0; f < F; ++f) x[f] = X[(size_t)s * F + f];
  mlp_forward_one(p, x, a1, a2, y);
  Y[s] = y;
}

// Gradient of L = (1/n) sum_s (y_s - t_s)^2 accumulated into grad (zeroed by
// the caller); loss accumulated into *loss.
__global__ void __launch_bounds__(kMlpThreads)
    k_mlp_backward(const float* params, const float* X, const float* T, int n, float* grad,
                   float* loss) {
  __shared__ float p[kNP];
  __shared__ float g[kNP];
  __shared__ float lsum;
  for (int i = threadIdx.x; i < kNP; i += blockDim.x) {
    p[i] = params[i];
    g[i] = 0.f;
  }
  if (threadIdx.x == 0) lsum = 0.f;
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) {
    float x[F], a1[H], a2[H], y;
    for (int f = 0; f < F; ++f) x[f] = X[(size_t)s * F + f];
    mlp_forward_one(p, x, a1, a2, y);
    const float e = y - T[s];
    atomicAdd(&lsum, e * e / n);
    const float dy = 2.f * e / n;
    // Output layer.
    atomicAdd(&g[kB3], dy);
    float d2[H];
    for (int h = 0; h < H; ++h) {
      atomicAdd(&g[kW3 + h], dy * a2[h]);
      d2[h] = dy * p[kW3 + h] * (1.f - a2[h] * a2[h]);
    }
    // Hidden layer 2.
    float d1[H];
    for (int k = 0; k < H; ++k) d1[k] = 0.f;
    for (int h = 0; h < H; ++h) {
      atomicAdd(&g[kB2 + h], d2[h]);
      for (int k = 0; k < H; ++k) {
        atomicAdd(&g[kW2 + h * H + k], d2[h] * a1[k]);
        d1[k] = fmaf(d2[h], p[kW2 + h * H + k], d1[k]);
      }
    }
    // Hidden layer 1.
    for (int k = 0; k < H; ++k) {
      const float dk = d1[k] * (1.f - a1[k] * a1[k]);
      atomicAdd(&g[kB1 + k], dk);
      for (int f = 0; f < F; ++f) atomicAdd(&g[kW1 + k * F + f], dk * x[f]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kNP; i += blockDim.x)
    if (g[i] != 0.f) atomicAdd(&grad[i], g[i]);
  if (threadIdx.x == 0 && lsum != 0.f) atomicAdd(loss, lsum);
}

// Adam (Kingma & Ba 2015) with bias correction; step t counts from 1.
__global__ void k_adam(float* params, float* m, float* v, const float* grad, int t, float lr,
                       float b1, float b2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNP) return;
  const float gi = grad[i];
  m[i] = b1 * m[i] + (1.f - b1) * gi;
  v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
  const float mh = m[i] / (1.f - powf(b1, (float)t));
  const float vh = v[i] / (1.f - powf(b2, (float)t));
  params[i] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace sqs

struct sqs_predictor {
  float* params = nullptr;  // device
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  float* scratch = nullptr;  // X, T, Y staging and the loss
  size_t scratch_floats = 0;
  int step = 0;
  cudaStream_t stream = nullptr;
};

namespace {

bool ensure_scratch(sqs_predictor* p, size_t floats) {
  if (p->scratch_floats >= floats) return true;
  if (p->scratch) cudaFree(p->scratch);
  p->scratch = nullptr;
  if (cudaMalloc(&p->scratch, floats * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    p->scratch_floats = 0;
    return false;
  }
  p->scratch_floats = floats;
  return true;
}

// Xavier-style uniform initialisation from a 64-bit LCG (deterministic).
void init_params(std::vector<float>& w, uint64_t seed) {
  uint64_t s = seed * 6364136223846793005ull + 1442695040888963407ull;
  auto uni = [&]() {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return (float)((s >> 40) * (1.0 / 16777216.0)) * 2.f - 1.f;
  };
  using namespace sqs;
  const float a1 = std::sqrt(6.f / (F + H)), a2 = std::sqrt(6.f / (H + H)),
              a3 = std::sqrt(6.f / (H + 1));
  for (int i = 0; i < H * F; ++i) w[kW1 + i] = a1 * uni();
  for (int i = 0; i < H * H; ++i) w[kW2 + i] = a2 * uni();
  for (int i = 0; i < H; ++i) w[kW3 + i] = a3 * uni();
  for (int i = 0; i < H; ++i) w[kB1 + i] = w[kB2 + i] = 0.f;
  w[kB3] = 0.f;
}

}  // namespace

extern "C" {

sqs_status sqs_predictor_create(uint64_t seed, void* cuda_stream, sqs_predictor** out) {
  if (!out) return SQS_ERR_ARG;
  sqs_predictor* p = new sqs_predictor();
  p->stream = (cudaStream_t)cuda_stream;
  const size_t bytes = sqs::kNP * sizeof(float);
  if (cudaMalloc(&p->params, bytes) != cudaSuccess || cudaMalloc(&p->m, bytes) != cudaSuccess ||
      cudaMalloc(&p->v, bytes) != cudaSuccess || cudaMalloc(&p->grad, bytes) != cudaSuccess) {
    cudaGetLastError();
    sqs_predictor_destroy(p);
    return SQS_ERR_OOM;
  }
  std::vector<float> w(sqs::kNP);
  init_params(w, seed);
  cudaMemcpy(p->params, w.data(), bytes, cudaMemcpyHostToDevice);
  cudaMemset(p->m, 0, bytes);
  cudaMemset(p->v, 0, bytes);
  *out = p;
  return SQS_OK;
}

void sqs_predictor_destroy(sqs_predictor* p) {
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  cudaFree(p->params);
  cudaFree(p->m);
  cudaFree(p->v);
  cudaFree(p->grad);
  cudaFree(p->scratch);
  cudaGetLastError();
  delete p;
}

sqs_status sqs_predictor_get_params(const sqs_predictor* p, float* out) {
  if (!p || !out) return SQS_ERR_ARG;
  return cudaMemcpy(out, p->params, sqs::kNP * sizeof(float), cudaMemcpyDeviceToHost) ==
                 cudaSuccess
             ? SQS_OK
             : SQS_ERR_CUDA;
}

sqs_status sqs_predictor_set_params(sqs_predictor* p, const float* in) {
  if (!p || !in) return SQS_ERR_ARG;
  p->step = 0;
  cudaMemset(p->m, 0, sqs::kNP * sizeof(float));
  cudaMemset(p->v, 0, sqs::kNP * sizeof(float));
  return cudaMemcpy(p->params, in, sqs::kNP * sizeof(float), cudaMemcpyHostToDevice) ==
                 cudaSuccess
             ? SQS_OK
             : SQS_ERR_CUDA;
}

sqs_status sqs_predictor_predict(sqs_predictor* p, const float* X, uint32_t n, float* Y) {
  if (!p || (n && (!X || !Y))) return SQS_ERR_ARG;
  if (n == 0) return SQS_OK;
  if (!ensure_scratch(p, (size_t)n * (sqs::F + 1))) return SQS_ERR_OOM;
  float* dX = p->scratch;
  float* dY = dX + (size_t)n * sqs::F;
  cudaError_t e =
      cudaMemcpyAsync(dX, X, (size_t)n * sqs::F * sizeof(float), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) {
    sqs::k_mlp_forward<<<(n + sqs::kMlpThreads - 1) / sqs::kMlpThreads, sqs::kMlpThreads, 0,
                         p->stream>>>(p->params, dX, (int)n, dY);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Y, dY, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  return e == cudaSuccess ? SQS_OK : SQS_ERR_CUDA;
}

sqs_status sqs_predictor_gradient(sqs_predictor* p, const float* X, const float* T, uint32_t n,
                                  float* grad, float* loss) {
  if (!p || !n || !X || !T || !grad) return SQS_ERR_ARG;
  if (!ensure_scratch(p, (size_t)n * (sqs::F + 1) + 1)) return SQS_ERR_OOM;
  float* dX = p->scratch;
  float* dT = dX + (size_t)n * sqs::F;
  float* dL = dT + n;
  cudaError_t e =
      cudaMemcpyAsync(dX, X, (size_t)n * sqs::F * sizeof(float), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dT, T, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->grad, 0, sqs::kNP * sizeof(float), p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(dL, 0, sizeof(float), p->stream);
  if (e == cudaSuccess) {
    sqs::k_mlp_backward<<<(n + sqs::kMlpThreads - 1) / sqs::kMlpThreads, sqs::kMlpThreads, 0,
                          p->stream>>>(p->params, dX, dT, (int)n, p->grad, dL);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(grad, p->grad, sqs::kNP * sizeof(float), cudaMemcpyDeviceToHost,
                        p->stream);
  float l = 0.f;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&l, dL, sizeof(float), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (loss) *loss = l;
  return e == cudaSuccess ? SQS_OK : SQS_ERR_CUDA;
}

sqs_status sqs_predictor_train(sqs_predictor* p, const float* X, const float* T, uint32_t n,
                               uint32_t epochs, uint32_t batch, float lr, float* final_loss) {
  if (!p || !n || !X || !T || batch == 0 || !(lr > 0.f)) return SQS_ERR_ARG;
  if (!ensure_scratch(p, (size_t)n * (sqs::F + 1) + 1)) return SQS_ERR_OOM;
  float* dX = p->scratch;
  float* dT = dX + (size_t)n * sqs::F;
  float* dL = dT + n;
  cudaError_t e =
      cudaMemcpyAsync(dX, X, (size_t)n * sqs::F * sizeof(float), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dT, T, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, p->stream);
  for (uint32_t ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (uint32_t off = 0; off < n && e == cudaSuccess; off += batch) {
      const uint32_t nb = n - off < batch ? n - off : batch;
      cudaMemsetAsync(p->grad, 0, sqs::kNP * sizeof(float), p->stream);
      cudaMemsetAsync(dL, 0, sizeof(float), p->stream);
      sqs::k_mlp_backward<<<(nb + sqs::kMlpThreads - 1) / sqs::kMlpThreads, sqs::kMlpThreads, 0,
                            p->stream>>>(p->params, dX + (size_t)off * sqs::F, dT + off, (int)nb,
                                         p->grad, dL);
      p->step++;
      sqs::k_adam<<<(sqs::kNP + 255) / 256, 256, 0, p->stream>>>(
          p->params, p->m, p->v, p->grad, p->step, lr, 0.9f, 0.999f, 1e-8f);
      e = cudaGetLastError();
    }
  }
  // Loss over the whole set with the final weights.
  if (e == cudaSuccess) {
    cudaMemsetAsync(p->grad, 0, sqs::kNP * sizeof(float), p->stream);
    cudaMemsetAsync(dL, 0, sizeof(float), p->stream);
    sqs::k_mlp_backward<<<(n + sqs::kMlpThreads - 1) / sqs::kMlpThreads, sqs::kMlpThreads, 0,
                          p->stream>>>(p->params, dX, dT, (int)n, p->grad, dL);
    e = cudaGetLastError();
  }
  float l = 0.f;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&l, dL, sizeof(float), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (final_loss) *final_loss = l;
  return e == cudaSuccess ? SQS_OK : SQS_ERR_CUDA;
}

}  // extern "C"
