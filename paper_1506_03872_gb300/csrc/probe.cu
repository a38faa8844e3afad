// Memory-system probes (the paper has no counterpart): the random-access
// rates that bound the sampler.  A diamond's draws end in a handful of
// random 32-byte sectors of the tables and, for 0/1 inputs, a random 64-bit
// atomic on the hash, so the ceilings of those kernels are the GPU's random
// sector gather rate and random atomic rate over buffers of the tables'
// and the hash's sizes, not its streaming copy bandwidth.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mad_internal.cuh"

namespace mad {
namespace {

constexpr int kProbeBlock = 256;
constexpr int kInFlight = 8;      // independent accesses per thread per step

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  // SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA'14).
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__device__ __forceinline__ uint64_t pick(uint64_t seed, uint64_t r, uint64_t n) {
  return __umul64hi(mix64(seed ^ r), n);   // uniform in [0, n)
}

// count reads of 4 bytes, each from a uniformly random 32-byte sector.
__global__ void __launch_bounds__(kProbeBlock) k_probe_gather(const uint32_t* __restrict__ table,
                                                              uint64_t sectors, uint64_t count,
                                                              uint64_t seed,
                                                              unsigned long long* sink) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t acc = 0;
  for (uint64_t r0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r0 < count;
       r0 += stride * kInFlight) {
    uint32_t v[kInFlight];
#pragma unroll
    for (int q = 0; q < kInFlight; ++q) {
      const uint64_t r = r0 + (uint64_t)q * stride;
      v[q] = r < count ? __ldg(table + 8 * pick(seed, r, sectors)) : 0u;
    }
#pragma unroll
    for (int q = 0; q < kInFlight; ++q) acc += v[q];
  }
  if (acc == 0x9E3779B9u) sink[0] = acc;   // keeps the loads; practically never taken
}

// count 64-bit atomics on uniformly random words: mode 0 adds (no value
// returned: a reduction), mode 1 compare-and-swaps and uses the old value
// (a round trip, as a hash insert's key claim).
__global__ void __launch_bounds__(kProbeBlock) k_probe_atomic(unsigned long long* table,
                                                              uint64_t words, uint64_t count,
                                                              uint64_t seed, int mode,
                                                              unsigned long long* sink) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long acc = 0;
  for (uint64_t r0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r0 < count;
       r0 += stride * kInFlight) {
    unsigned long long old[kInFlight];
#pragma unroll
    for (int q = 0; q < kInFlight; ++q) {
      const uint64_t r = r0 + (uint64_t)q * stride;
      old[q] = 0;
      if (r < count) {
        unsigned long long* w = table + pick(seed, r, words);
        if (mode == 0)
          atomicAdd(w, 1ull);
        else
          old[q] = atomicCAS(w, 0ull, r + 1);
      }
    }
#pragma unroll
    for (int q = 0; q < kInFlight; ++q) acc += old[q];
  }
  if (mode != 0 && acc == 0x9E3779B97F4A7C15ull) sink[0] = acc;
}

template <class K>
unsigned probe_grid(K kernel, uint64_t count) {
  int dev = 0, sms = 152, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kProbeBlock, 0);
  if (per_sm < 1) per_sm = 1;
  uint64_t blocks = (uint64_t)sms * per_sm;
  const uint64_t need = (count + kProbeBlock - 1) / kProbeBlock;
  if (blocks > need) blocks = need ? need : 1;
  return (unsigned)blocks;
}

}  // namespace
}  // namespace mad

using namespace mad;

mad_status mad_probe_gather(const void* table_dev, uint64_t bytes, uint64_t count, uint64_t seed,
                            void* sink_dev, mad_stream stream) {
  if (!table_dev || !sink_dev || bytes < 32 || (bytes & 31) || ((uintptr_t)table_dev & 31))
    return MAD_ERR_ARG;
  if (count == 0) return MAD_OK;
  k_probe_gather<<<probe_grid(k_probe_gather, count), kProbeBlock, 0, (cudaStream_t)stream>>>(
      (const uint32_t*)table_dev, bytes / 32, count, seed, (unsigned long long*)sink_dev);
  return cuda_status(cudaGetLastError());
}

mad_status mad_probe_atomics(void* table_dev, uint64_t bytes, uint64_t count, uint32_t mode,
                             uint64_t seed, void* sink_dev, mad_stream stream) {
  if (!table_dev || !sink_dev || bytes < 8 || (bytes & 7) || ((uintptr_t)table_dev & 7) ||
      mode > 1)
    return MAD_ERR_ARG;
  if (count == 0) return MAD_OK;
  k_probe_atomic<<<probe_grid(k_probe_atomic, count), kProbeBlock, 0, (cudaStream_t)stream>>>(
      (unsigned long long*)table_dev, bytes / 8, count, seed, (int)mode,
      (unsigned long long*)sink_dev);
  return cuda_status(cudaGetLastError());
}
