// Device-side building blocks: counter-based RNG, inverse-CDF searches,
// fixed-order reductions and the open-addressing hash.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mad_internal.cuh"

namespace mad {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies; the key advances by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// The four 64-bit uniforms of diamond ell: counter (ell_lo, ell_hi, 0, blk).
struct Uniforms {
  unsigned long long u0, u1, u2, u3;
};

__device__ __forceinline__ Uniforms diamond_uniforms(unsigned long long seed,
                                                     unsigned long long ell) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const uint4 b0 = philox4x32_10(make_uint4((uint32_t)ell, (uint32_t)(ell >> 32), 0u, 0u), key);
  const uint4 b1 = philox4x32_10(make_uint4((uint32_t)ell, (uint32_t)(ell >> 32), 0u, 1u), key);
  Uniforms u;
  u.u0 = ((unsigned long long)b0.y << 32) | b0.x;
  u.u1 = ((unsigned long long)b0.w << 32) | b0.z;
  u.u2 = ((unsigned long long)b1.y << 32) | b1.x;
  u.u3 = ((unsigned long long)b1.w << 32) | b1.z;
  return u;
}

// floor(u * total / 2^64).
__device__ __forceinline__ unsigned long long draw_target(unsigned long long u,
                                                          unsigned long long total) {
  return __umul64hi(u, total);
}

// First position p in [0, len) with prefix[p] > target (masking the sign
// bit of row tables).  Clamped to len-1 when the table is inconsistent.
__device__ __forceinline__ int64_t search_u64(const uint64_t* __restrict__ prefix, int64_t len,
                                              unsigned long long target, bool* bad) {
  int64_t lo = 0, hi = len;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg((const unsigned long long*)prefix + mid) > target)
      hi = mid;
    else
      lo = mid + 1;
  }
  if (lo >= len) {
    *bad = true;
    lo = len - 1;
  }
  return lo;
}

__device__ __forceinline__ int64_t search_u32(const uint32_t* __restrict__ prefix, int64_t len,
                                              uint32_t target, uint32_t mask, bool* bad) {
  int64_t lo = 0, hi = len;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((__ldg(prefix + mid) & mask) > target)
      hi = mid;
    else
      lo = mid + 1;
  }
  if (lo >= len) {
    *bad = true;
    lo = len - 1;
  }
  return lo;
}

// The same searches through a coarse index (coarse[g] = prefix entry
// min((g+1) 2^lg, len) - 1): the block whose last entry first exceeds the
// target holds the answer, so the result equals the full search.
__device__ __forceinline__ int64_t search_coarse_u64(const uint64_t* coarse, int64_t nc,
                                                     const uint64_t* __restrict__ prefix,
                                                     int64_t len, int lg,
                                                     unsigned long long target, bool* bad) {
  int64_t lo = 0, hi = nc;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((unsigned long long)coarse[mid] > target)
      hi = mid;
    else
      lo = mid + 1;
  }
  if (lo >= nc) {
    *bad = true;
    lo = nc - 1;
  }
  const int64_t base = lo << lg;
  const int64_t wlen = (len - base) < (1ll << lg) ? (len - base) : (1ll << lg);
  return base + search_u64(prefix + base, wlen, target, bad);
}

__device__ __forceinline__ int64_t search_coarse_u32(const uint32_t* coarse, int64_t nc,
                                                     const uint32_t* __restrict__ prefix,
                                                     int64_t len, int lg, uint32_t target,
                                                     uint32_t mask, bool* bad) {
  int64_t lo = 0, hi = nc;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (coarse[mid] > target)
      hi = mid;
    else
      lo = mid + 1;
  }
  if (lo >= nc) {
    *bad = true;
    lo = nc - 1;
  }
  const int64_t base = lo << lg;
  const int64_t wlen = (len - base) < (1ll << lg) ? (len - base) : (1ll << lg);
  return base + search_u32(prefix + base, wlen, target, mask, bad);
}

// Sorted-list membership (0/1 CSR closure test).
__device__ __forceinline__ bool contains_sorted(const int32_t* __restrict__ list, int64_t len,
                                                int32_t value) {
  int64_t lo = 0, hi = len;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    const int32_t v = __ldg(list + mid);
    if (v < value)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo < len && __ldg(list + lo) == value;
}

// Exponent of a positive finite FP32 value (floor(log2 x)), from its bits.
__device__ __forceinline__ int ilogb_pos(float x) {
  const uint32_t b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xFF);
  if (e != 0) return e - 127;
  // subnormal: value = mantissa * 2^-149
  const uint32_t mant = b & 0x7FFFFF;
  return (31 - __clz(mant)) - 149;
}

// 2^e as a double, for |e| <= 1022.
__device__ __forceinline__ double pow2d(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// ---------------------------------------------------------------------------
// Open-addressing hash for X: 64-bit keys (EMPTY_KEY = free), int64 values,
// linear probing from a splitmix64-finalised slot.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Linear probing from `slot`, wrapping at cap.  Returns 0 when the probe
// limit is hit, 1 when the key existed, 2 when this call created it.
__device__ __forceinline__ int hash_add_from(unsigned long long* __restrict__ keys,
                                             long long* __restrict__ vals, uint64_t cap,
                                             uint64_t slot, uint32_t max_probe,
                                             unsigned long long key, long long v) {
  for (uint32_t probe = 0; probe < max_probe; ++probe) {
    // Claim-or-match in one atomic: the slot is ours when it was empty or
    // already held the key.
    const unsigned long long prev = atomicCAS(keys + slot, EMPTY_KEY, key);
    if (prev == EMPTY_KEY || prev == key) {
      atomicAdd((unsigned long long*)vals + slot, (unsigned long long)v);
      return prev == EMPTY_KEY ? 2 : 1;
    }
    slot = (slot + 1 == cap) ? 0 : slot + 1;
  }
  return 0;
}

// First slot probed for key = (a << 32) | b.
__device__ __forceinline__ uint64_t home_slot(const SampleParams& p, unsigned long long key) {
  if (p.regioned) {
    const uint32_t a = (uint32_t)(key >> 32);
    const unsigned long long r0 = p.hreg[a];
    const unsigned long long size = p.hreg[a + 1] - r0;  // a power of two
    return r0 + (mix64(key) & (size - 1));
  }
  return mix64(key) & p.hmask;
}

__device__ __forceinline__ int hash_add(const SampleParams& p, unsigned long long key, long long v) {
  return hash_add_from(p.hkeys, p.hvals, p.hcap, home_slot(p, key), p.max_probe, key, v);
}

}  // namespace mad
