// Cheap statistics of an instance for the learned budget predictor: sizes,
// ||W||_1, the largest row and column 2-norms (a Cauchy-Schwarz stand-in
// for Theorem 2's tau) and the concentration of the row weights of T1.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>

#include "mad_device.cuh"
#include "mad_internal.cuh"

namespace mad {
namespace {

struct FeatScratch {
  unsigned int max_a2_bits;      // largest row 2-norm of A (FP32 bits)
  unsigned int max_b2_bits;      // largest column 2-norm of B
  unsigned long long max_q;      // largest row weight of T1 (integer)
  double sum_q2;                 // sum of squared row weights
  unsigned int counts_pad;
};

template <typename T>
__device__ __forceinline__ float as_f32(T v) { return (float)v; }

// Largest squared row norm of dense A: one warp per row.
template <typename T>
__global__ void __launch_bounds__(256)
k_feat_rows(const T* __restrict__ A, int64_t m, int64_t d, int64_t lda, FeatScratch* fs) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float best = 0.0f;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
    float s = 0.0f;
    for (int64_t k = lane; k < d; k += 32) {
      const float v = as_f32(A[i * lda + k]);
      s = __fmaf_rn(v, v, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    best = fmaxf(best, s);
  }
  if (lane == 0 && best > 0.0f) atomicMax(&fs->max_a2_bits, __float_as_uint(sqrtf(best)));
}

// Largest column norm of dense B (d x n): one thread per column.
template <typename T>
__global__ void __launch_bounds__(256)
k_feat_cols(const T* __restrict__ B, int64_t d, int64_t n, int64_t ldb, FeatScratch* fs) {
  float best = 0.0f;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int64_t k = 0; k < d; ++k) {
      const float v = as_f32(B[k * ldb + j]);
      s = __fmaf_rn(v, v, s);
    }
    best = fmaxf(best, s);
  }
  if (best > 0.0f) atomicMax(&fs->max_b2_bits, __float_as_uint(sqrtf(best)));
}

// 0/1 CSR: the largest row degree of A, and column counts of B.
__global__ void __launch_bounds__(256)
k_feat_deg(const int64_t* __restrict__ ptr, int64_t rows, FeatScratch* fs) {
  unsigned long long best = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long deg = (unsigned long long)(ptr[i + 1] - ptr[i]);
    best = deg > best ? deg : best;
  }
  if (best) atomicMax(&fs->max_a2_bits, __float_as_uint(sqrtf((float)best)));
}

__global__ void __launch_bounds__(256)
k_feat_col_hist(const int32_t* __restrict__ col, int64_t nnz, unsigned int* __restrict__ cnt) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + col[e], 1u);
}

__global__ void __launch_bounds__(256)
k_feat_col_max(const unsigned int* __restrict__ cnt, int64_t n, FeatScratch* fs) {
  unsigned int best = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    best = cnt[j] > best ? cnt[j] : best;
  if (best) atomicMax(&fs->max_b2_bits, __float_as_uint(sqrtf((float)best)));
}

// Row weights of T1 (its increments): largest and sum of squares.
__global__ void __launch_bounds__(256)
k_feat_t1(const uint64_t* __restrict__ T1, int64_t m, FeatScratch* fs) {
  __shared__ double part[256];
  double s2 = 0.0;
  unsigned long long best = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long q = T1[i] - (i ? T1[i - 1] : 0ull);
    s2 += (double)q * (double)q;
    best = q > best ? q : best;
  }
  part[threadIdx.x] = s2;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(&fs->sum_q2, part[0]);
  if (best) atomicMax(&fs->max_q, best);
}

unsigned grid_for_rows(int64_t rows) {
  const int64_t b = (rows + 255) / 256;
  return (unsigned)(b < 152 * 8 ? (b ? b : 1) : 152 * 8);
}

}  // namespace
}  // namespace mad

using namespace mad;

extern "C" mad_status mad_budget_features(mad_ctx* ctx, float* features_host, mad_stream stream) {
  if (!ctx || !features_host) return MAD_ERR_ARG;
  if (!ctx->built) return MAD_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t hist_bytes = ctx->integer ? (size_t)ctx->n * sizeof(unsigned int) : 0;
  mad_status rs = ensure_scratch(ctx, 256 + hist_bytes, st);
  if (rs != MAD_OK) return rs;
  FeatScratch* fs = (FeatScratch*)ctx->scratch;
  cudaMemsetAsync(fs, 0, 256 + hist_bytes, st);
  if (ctx->integer) {
    k_feat_deg<<<grid_for_rows(ctx->m), 256, 0, st>>>(ctx->A.rowptr, ctx->m, fs);
    unsigned int* cnt = (unsigned int*)((char*)ctx->scratch + 256);
    k_feat_col_hist<<<grid_for_rows((int64_t)ctx->nnz_b), 256, 0, st>>>(ctx->B.colidx,
                                                                        (int64_t)ctx->nnz_b, cnt);
    k_feat_col_max<<<grid_for_rows(ctx->n), 256, 0, st>>>(cnt, ctx->n, fs);
    count_launch(ctx, 3);
  } else {
    if (ctx->A.dt == MAD_F64)
      k_feat_rows<double><<<grid_for_rows(ctx->m * 32), 256, 0, st>>>(
          (const double*)ctx->A.values, ctx->m, ctx->d, ctx->A.ld, fs);
    else
      k_feat_rows<float><<<grid_for_rows(ctx->m * 32), 256, 0, st>>>(
          (const float*)ctx->A.values, ctx->m, ctx->d, ctx->A.ld, fs);
    if (ctx->B.dt == MAD_F64)
      k_feat_cols<double><<<grid_for_rows(ctx->n), 256, 0, st>>>((const double*)ctx->B.values,
                                                                 ctx->d, ctx->n, ctx->B.ld, fs);
    else
      k_feat_cols<float><<<grid_for_rows(ctx->n), 256, 0, st>>>((const float*)ctx->B.values, ctx->d,
                                                                ctx->n, ctx->B.ld, fs);
    count_launch(ctx, 2);
  }
  k_feat_t1<<<grid_for_rows(ctx->m), 256, 0, st>>>(ctx->T1, ctx->m, fs);
  count_launch(ctx);
  FeatScratch h;
  cudaMemcpyAsync(&h, fs, sizeof(h), cudaMemcpyDeviceToHost, st);
  if ((rs = cuda_status(cudaStreamSynchronize(st))) != MAD_OK) return rs;
  float a2, b2;
  std::memcpy(&a2, &h.max_a2_bits, sizeof(float));
  std::memcpy(&b2, &h.max_b2_bits, sizeof(float));
  const double w1 = ctx->integer ? (double)ctx->t1_total : std::ldexp((double)ctx->t1_total, -ctx->e1);
  const double tot = (double)ctx->t1_total;
  auto lg = [](double v) { return (float)std::log10(v > 1e-300 ? v : 1e-300); };
  features_host[0] = lg((double)ctx->m);
  features_host[1] = lg((double)ctx->n);
  features_host[2] = lg((double)ctx->d);
  features_host[3] = lg((double)ctx->nnz_a);
  features_host[4] = lg((double)ctx->nnz_b);
  features_host[5] = ctx->integer ? 1.0f : 0.0f;
  features_host[6] = lg(w1);
  features_host[7] = lg((double)a2);
  features_host[8] = lg((double)b2);
  features_host[9] = lg(h.sum_q2 / (tot * tot));
  features_host[10] = lg((double)h.max_q / tot);
  features_host[11] = features_host[6] - 2.0f * (features_host[7] + features_host[8]);
  return MAD_OK;
}
