// Exclusive prefix sums over device arrays (three launches: per-chunk sums,
// chunk offsets, chunk-local scans).  Integer sums, so the result does not
// depend on the blocking.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mad_internal.cuh"

namespace mad {
namespace {

constexpr int kChunk = 2048;  // 256 threads x 8 elements

template <typename T>
__device__ __forceinline__ T warp_inclusive(T v, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T o = __shfl_up_sync(0xFFFFFFFFu, v, off);
    if (lane >= off) v += o;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T block_exclusive(T v, T* warp_tot, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T inc = warp_inclusive(v, lane);
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const T t = lane < 8 ? warp_tot[lane] : (T)0;
    const T ti = warp_inclusive(t, lane);
    if (lane < 8) warp_tot[lane] = ti - t;
    if (lane == 7) warp_tot[8] = ti;
  }
  __syncthreads();
  const T out = warp_tot[warp] + inc - v;
  *total = warp_tot[8];
  __syncthreads();
  return out;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_chunk_sums(const T* __restrict__ in, uint64_t n, T* __restrict__ partial) {
  __shared__ T warp_tot[9];
  const uint64_t base = (uint64_t)blockIdx.x * kChunk + threadIdx.x * 8;
  T acc = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (base + c < n) acc += in[base + c];
  T total;
  block_exclusive(acc, warp_tot, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// Exclusive scan of the chunk sums by one block, tile by tile.
template <typename T>
__global__ void __launch_bounds__(256)
k_chunk_offsets(T* __restrict__ partial, uint64_t chunks, T* __restrict__ total_out) {
  __shared__ T warp_tot[9];
  __shared__ T carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t base = 0; base < chunks; base += 256) {
    const uint64_t idx = base + threadIdx.x;
    const T v = idx < chunks ? partial[idx] : (T)0;
    T tile;
    const T ex = block_exclusive(v, warp_tot, &tile);
    if (idx < chunks) partial[idx] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tile;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total_out = carry;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_chunk_write(const T* __restrict__ in, uint64_t n, const T* __restrict__ offset,
              T* __restrict__ out) {
  __shared__ T warp_tot[9];
  const uint64_t base = (uint64_t)blockIdx.x * kChunk + threadIdx.x * 8;
  T v[8], acc = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    v[c] = (base + c < n) ? in[base + c] : (T)0;
    acc += v[c];
  }
  T total;
  T run = offset[blockIdx.x] + block_exclusive(acc, warp_tot, &total);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (base + c < n) out[base + c] = run;
    run += v[c];
  }
}

template <typename T>
mad_status scan_impl(mad_ctx* ctx, const T* in, T* out, uint64_t n, T* partial,
                     cudaStream_t st) {
  const uint64_t chunks = (n + kChunk - 1) / kChunk;
  if (n == 0) return cuda_status(cudaMemsetAsync(out, 0, sizeof(T), st));
  k_chunk_sums<T><<<(unsigned)chunks, 256, 0, st>>>(in, n, partial);
  k_chunk_offsets<T><<<1, 256, 0, st>>>(partial, chunks, out + n);
  k_chunk_write<T><<<(unsigned)chunks, 256, 0, st>>>(in, n, partial, out);
  count_launch(ctx, 3);
  return cuda_status(cudaGetLastError());
}

}  // namespace

size_t scan_partial_elems(uint64_t n) { return (n + kChunk - 1) / kChunk + 1; }

mad_status scan_exclusive_u32(mad_ctx* ctx, const uint32_t* in, uint32_t* out, uint64_t n,
                              uint32_t* partial, cudaStream_t st) {
  return scan_impl<unsigned int>(ctx, (const unsigned int*)in, (unsigned int*)out, n,
                                 (unsigned int*)partial, st);
}

mad_status scan_exclusive_u64(mad_ctx* ctx, const uint64_t* in, uint64_t* out, uint64_t n,
                              uint64_t* partial, cudaStream_t st) {
  return scan_impl<unsigned long long>(ctx, (const unsigned long long*)in,
                                       (unsigned long long*)out, n,
                                       (unsigned long long*)partial, st);
}

}  // namespace mad
