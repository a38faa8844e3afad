// Learned budget predictor: a 3-layer perceptron (f -> 64 -> 64 -> 1, ReLU)
// that maps cheap statistics of an instance to log10 of the diamond budget
// reaching a target recall.  Weights are used in BF16 (FP32 master copies
// for training), activations and accumulation are FP32.  Theorem 2 of the
// paper (s grows as ||W||_1 / tau^2) motivates the features; the network
// learns the rest from recall curves the sampler itself produced.
//
// Training is full-batch Adam on a pinball (quantile) loss, which weighs a
// budget that falls short more than one that overshoots; the whole loop runs
// in one CTA (the data are a few hundred instances), so every reduction has
// one fixed order and a run is deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mad_internal.cuh"

namespace mad {
namespace {

constexpr int H = MAD_MLP_HIDDEN;   // hidden width
constexpr int kFMax = 32;           // largest feature count
constexpr int kNMax = 4096;         // largest training set

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

struct Layout {
  int f;
  int w1, b1, w2, b2, w3, b3, total;
};

__host__ __device__ inline Layout layout(int f) {
  Layout L;
  L.f = f;
  L.w1 = 0;
  L.b1 = L.w1 + H * f;
  L.w2 = L.b1 + H;
  L.b2 = L.w2 + H * H;
  L.w3 = L.b2 + H;
  L.b3 = L.w3 + H;
  L.total = L.b3 + 1;
  return L;
}

// Forward pass of one sample with BF16-rounded weights held in shared
// memory (w1s: H x f, w2s: H x H, w3s: H); writes both hidden layers.
__device__ __forceinline__ float forward(const float* x, int f, const float* w1s, const float* b1,
                                         const float* w2s, const float* b2, const float* w3s,
                                         float b3, float* h1, float* h2) {
  for (int h = 0; h < H; ++h) {
    float a = b1[h];
    for (int k = 0; k < f; ++k) a = __fmaf_rn(w1s[h * f + k], x[k], a);
    h1[h] = a > 0.0f ? a : 0.0f;
  }
  for (int h = 0; h < H; ++h) {
    float a = b2[h];
    for (int j = 0; j < H; ++j) a = __fmaf_rn(w2s[h * H + j], h1[j], a);
    h2[h] = a > 0.0f ? a : 0.0f;
  }
  float y = b3;
  for (int h = 0; h < H; ++h) y = __fmaf_rn(w3s[h], h2[h], y);
  return y;
}

// Full-batch training, one CTA.  Per epoch: forward and per-sample
// backward (hidden activations and their gradients to `act`), gradients
// summed over the samples in index order, one Adam step on the FP32 master
// parameters, BF16 copies refreshed.
__global__ void __launch_bounds__(256, 1)
k_mlp_train(float* __restrict__ P, const float* __restrict__ X, const float* __restrict__ y,
            int n, int f, int epochs, float lr, float quantile, float* __restrict__ loss_out,
            float* __restrict__ act, float* __restrict__ grad, float* __restrict__ m1,
            float* __restrict__ m2) {
  __shared__ float w1s[H * kFMax], w2s[H * H], w3s[H];
  __shared__ float red[256];
  const Layout L = layout(f);
  const int tid = threadIdx.x;
  for (int e = tid; e < L.total; e += blockDim.x) m1[e] = m2[e] = 0.0f;
  float b1p = 1.0f, b2p = 1.0f;   // beta powers
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int e = tid; e < H * f; e += blockDim.x) w1s[e] = bf16r(P[L.w1 + e]);
    for (int e = tid; e < H * H; e += blockDim.x) w2s[e] = bf16r(P[L.w2 + e]);
    for (int e = tid; e < H; e += blockDim.x) w3s[e] = bf16r(P[L.w3 + e]);
    __syncthreads();
    // per-sample forward and backward; act row s: h1 (H), h2 (H), d1 (H), d2 (H), g
    float loss = 0.0f;
    for (int s = tid; s < n; s += blockDim.x) {
      float* r = act + (size_t)s * (4 * H + 1);
      const float yh = forward(X + (size_t)s * f, f, w1s, P + L.b1, w2s, P + L.b2, w3s, P[L.b3],
                               r, r + H);
      const float err = y[s] - yh;
      loss += err > 0.0f ? quantile * err : (quantile - 1.0f) * err;
      const float g = (err > 0.0f ? -quantile : (err < 0.0f ? 1.0f - quantile : 0.0f)) / (float)n;
      r[4 * H] = g;
      for (int h = 0; h < H; ++h) r[3 * H + h] = r[H + h] > 0.0f ? g * w3s[h] : 0.0f;   // d2
      for (int j = 0; j < H; ++j) {
        float a = 0.0f;
        for (int h = 0; h < H; ++h) a = __fmaf_rn(w2s[h * H + j], r[3 * H + h], a);
        r[2 * H + j] = r[j] > 0.0f ? a : 0.0f;                                           // d1
      }
    }
    red[tid] = loss;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (tid < o) red[tid] += red[tid + o];
      __syncthreads();
    }
    if (tid == 0 && loss_out) loss_out[ep] = red[0] / (float)n;
    // gradients, each summed over the samples in index order
    for (int e = tid; e < L.total; e += blockDim.x) {
      float a = 0.0f;
      if (e < L.b1) {                       // W1[h][k]
        const int h = e / f, k = e % f;
        for (int s = 0; s < n; ++s) a = __fmaf_rn(act[(size_t)s * (4 * H + 1) + 2 * H + h], X[(size_t)s * f + k], a);
      } else if (e < L.w2) {                // b1[h]
        const int h = e - L.b1;
        for (int s = 0; s < n; ++s) a += act[(size_t)s * (4 * H + 1) + 2 * H + h];
      } else if (e < L.b2) {                // W2[h][j]
        const int h = (e - L.w2) / H, j = (e - L.w2) % H;
        for (int s = 0; s < n; ++s) {
          const float* r = act + (size_t)s * (4 * H + 1);
          a = __fmaf_rn(r[3 * H + h], r[j], a);
        }
      } else if (e < L.w3) {                // b2[h]
        const int h = e - L.b2;
        for (int s = 0; s < n; ++s) a += act[(size_t)s * (4 * H + 1) + 3 * H + h];
      } else if (e < L.b3) {                // w3[h]
        const int h = e - L.w3;
        for (int s = 0; s < n; ++s) {
          const float* r = act + (size_t)s * (4 * H + 1);
          a = __fmaf_rn(r[4 * H], r[H + h], a);
        }
      } else {                              // b3
        for (int s = 0; s < n; ++s) a += act[(size_t)s * (4 * H + 1) + 4 * H];
      }
      grad[e] = a;
    }
    __syncthreads();
    b1p *= beta1;
    b2p *= beta2;
    for (int e = tid; e < L.total; e += blockDim.x) {
      const float g = grad[e];
      m1[e] = beta1 * m1[e] + (1.0f - beta1) * g;
      m2[e] = beta2 * m2[e] + (1.0f - beta2) * g * g;
      const float mh = m1[e] / (1.0f - b1p), vh = m2[e] / (1.0f - b2p);
      P[e] -= lr * mh / (sqrtf(vh) + eps);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
k_mlp_predict(const float* __restrict__ P, const float* __restrict__ X, int n, int f,
              float* __restrict__ y) {
  __shared__ float w1s[H * kFMax], w2s[H * H], w3s[H];
  const Layout L = layout(f);
  for (int e = threadIdx.x; e < H * f; e += blockDim.x) w1s[e] = bf16r(P[L.w1 + e]);
  for (int e = threadIdx.x; e < H * H; e += blockDim.x) w2s[e] = bf16r(P[L.w2 + e]);
  for (int e = threadIdx.x; e < H; e += blockDim.x) w3s[e] = bf16r(P[L.w3 + e]);
  __syncthreads();
  float h1[H], h2[H];
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
    y[s] = forward(X + (size_t)s * f, f, w1s, P + L.b1, w2s, P + L.b2, w3s, P[L.b3], h1, h2);
}

}  // namespace
}  // namespace mad

using namespace mad;

extern "C" {

mad_status mad_mlp_train(mad_ctx* ctx, float* params_dev, const float* X_dev, const float* y_dev,
                         uint32_t n, uint32_t f, uint32_t epochs, float lr, float quantile,
                         float* loss_dev, mad_stream stream) {
  if (!ctx || !params_dev || !X_dev || !y_dev || n == 0 || n > (uint32_t)kNMax || f == 0 ||
      f > (uint32_t)kFMax || !(lr > 0.0f) || !(quantile > 0.0f && quantile < 1.0f))
    return MAD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout L = layout((int)f);
  const size_t act = (size_t)n * (4 * H + 1), params = (size_t)L.total;
  mad_status rs = ensure_scratch(ctx, (act + 3 * params) * sizeof(float) + 1024, st);
  if (rs != MAD_OK) return rs;
  float* base = (float*)ctx->scratch;
  k_mlp_train<<<1, 256, 0, st>>>(params_dev, X_dev, y_dev, (int)n, (int)f, (int)epochs, lr,
                                 quantile, loss_dev, base, base + act, base + act + params,
                                 base + act + 2 * params);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

mad_status mad_mlp_predict(const float* params_dev, const float* X_dev, uint32_t n, uint32_t f,
                           float* y_dev, mad_stream stream) {
  if (!params_dev || !X_dev || !y_dev || f == 0 || f > (uint32_t)kFMax) return MAD_ERR_ARG;
  if (n == 0) return MAD_OK;
  const unsigned blocks = (n + 255) / 256 < 152 ? (n + 255) / 256 : 152;
  k_mlp_predict<<<blocks, 256, 0, (cudaStream_t)stream>>>(params_dev, X_dev, (int)n, (int)f, y_dev);
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
