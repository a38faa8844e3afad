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

// Uniforms of Philox blocks 2 and 3 of diamond ell: the segment-level
// uniforms of two-level alias draws (index q of (i, k, j, k') takes u_q of
// diamond_uniforms first and the q-th of these second).
__device__ __forceinline__ Uniforms alias_uniforms(unsigned long long seed, unsigned long long ell) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const uint4 b2 = philox4x32_10(make_uint4((uint32_t)ell, (uint32_t)(ell >> 32), 0u, 2u), key);
  const uint4 b3 = philox4x32_10(make_uint4((uint32_t)ell, (uint32_t)(ell >> 32), 0u, 3u), key);
  Uniforms u;
  u.u0 = ((unsigned long long)b2.y << 32) | b2.x;
  u.u1 = ((unsigned long long)b2.w << 32) | b2.z;
  u.u2 = ((unsigned long long)b3.y << 32) | b3.x;
  u.u3 = ((unsigned long long)b3.w << 32) | b3.z;
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
  // Row lengths are below 2^31: 32-bit indices.
  int lo = 0, hi = (int)len;
  while (lo < hi) {
    const int mid = (int)(((unsigned)lo + (unsigned)hi) >> 1);
    if ((__ldg(prefix + mid) & mask) > target)
      hi = mid;
    else
      lo = mid + 1;
  }
  if (lo >= (int)len) {
    *bad = true;
    lo = (int)len - 1;
  }
  return lo;
}

// Branch-free upper bound with a fixed number of steps (floor(log2 len) +
// 1, the same for every lane of a row length): the number of entries <=
// target, i.e. the position of the first entry above it.
__device__ __forceinline__ int ub_steps(int len) { return 32 - __clz(len); }

__device__ __forceinline__ int ub_u32(const uint32_t* __restrict__ P, int len, uint32_t target,
                                      uint32_t mask) {
  int pos = 0;
  for (int step = 1 << (31 - __clz(len)); step > 0; step >>= 1) {
    const int np = pos + step;
    const uint32_t v = __ldg(P + (np <= len ? np : len) - 1) & mask;
    pos = (np <= len && v <= target) ? np : pos;
  }
  return pos;
}

// Upper bound in a long row through its guide: bucket b = target >> sh
// holds the answer between guide entries b and b + 1, and the prefix
// entries between those positions are counted (a window of 4, else of 16,
// else a binary search over the bucket's range).  Same result as ub_u32
// over the whole row.
__device__ __forceinline__ int ub_guided_u32(const uint32_t* __restrict__ P,
                                             const uint32_t* __restrict__ G, int sh,
                                             uint32_t target, uint32_t mask = 0xFFFFFFFFu) {
  const uint32_t b = target >> sh;
  const int lo = (int)__ldg(G + b), hi = (int)__ldg(G + b + 1);
  if (hi - lo <= 4) {
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = lo + q;
      if (e < hi) cnt += ((__ldg(P + e) & mask) <= target) ? 1 : 0;
    }
    return lo + cnt;
  }
  if (hi - lo <= 16) {
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = lo + q;
      if (e < hi) cnt += ((__ldg(P + e) & mask) <= target) ? 1 : 0;
    }
    return lo + cnt;
  }
  return lo + ub_u32(P + lo, hi - lo, target, mask);
}

// The same for a 64-bit prefix (T1): bucket b = target >> sh.
__device__ __forceinline__ int64_t ub_guided_u64(const uint64_t* __restrict__ P, int64_t len,
                                                 const uint32_t* __restrict__ G, int sh,
                                                 unsigned long long target) {
  const unsigned long long b = target >> sh;
  const int64_t lo = (int64_t)__ldg(G + b), hi = (int64_t)__ldg(G + b + 1);
  if (hi - lo <= 4) {
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t e = lo + q;
      if (e < hi) cnt += (__ldg(P + e) <= target) ? 1 : 0;
    }
    return lo + cnt;
  }
  if (hi - lo <= 16) {
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int64_t e = lo + q;
      if (e < hi) cnt += (__ldg(P + e) <= target) ? 1 : 0;
    }
    return lo + cnt;
  }
  int64_t pos = lo, n = hi - lo;   // first entry above target in [lo, hi)
  while (n > 0) {
    const int64_t half = n >> 1;
    if (__ldg(P + pos + half) <= target) {
      pos += half + 1;
      n -= half + 1;
    } else {
      n = half;
    }
  }
  return pos < len ? pos : len;
}

// Two searches over rows of the same length at once (independent loads).
__device__ __forceinline__ void ub2_u32(const uint32_t* __restrict__ P, const uint32_t* __restrict__ Q,
                                        int len, uint32_t tp, uint32_t tq, uint32_t mask, int* op,
                                        int* oq) {
  int a = 0, b = 0;
  for (int step = 1 << (31 - __clz(len)); step > 0; step >>= 1) {
    const int na = a + step, nb = b + step;
    const uint32_t va = __ldg(P + (na <= len ? na : len) - 1) & mask;
    const uint32_t vb = __ldg(Q + (nb <= len ? nb : len) - 1) & mask;
    a = (na <= len && va <= tp) ? na : a;
    b = (nb <= len && vb <= tq) ? nb : b;
  }
  *op = a;
  *oq = b;
}

// A length known only on the device: min(cap, *n_dev), or cap itself when
// there is no device count.
__device__ __forceinline__ unsigned long long dev_len(unsigned long long cap,
                                                      const unsigned long long* n_dev) {
  if (!n_dev) return cap;
  const unsigned long long n = *n_dev;
  return n < cap ? n : cap;
}

// 2^e as an FP32 value, -126 <= e <= 127.
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// b * 2^F rounded to the nearest integer, ties to even, as int64 (callers
// keep |b * 2^F| < 2^63).  Scaling an FP32 value by a power of two is exact
// while the product stays a normal number, so the product is formed exactly
// (in two steps when 2^F itself is outside the normal range, each step
// keeping its result normal) and converted once with round-to-nearest-even.
// A product below 2^-126 in magnitude rounds to 0 whatever its last bits.
__device__ __forceinline__ long long fixed_point(float b, int F) {
  float x;
  if (F > 127) {
    x = (b * pow2f(127)) * pow2f(min(F - 127, 127));
  } else if (F < -126) {
    x = (b * pow2f(-126)) * pow2f(max(F + 126, -126));
  } else {
    x = b * pow2f(F);
  }
  return __float2ll_rn(x);
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
// 32-bit finaliser of MurmurHash3 (Appleby): spreads a column index over a
// home region (the row is fixed within a region, so the column suffices).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Linear probing from `slot`, wrapping at cap, four slots per round trip:
// the keys of the 32-byte group holding `slot` are read with two 16-byte
// loads, and the first slot of the group (from `slot` on) that is empty or
// holds the key is picked without branching (lanes of a warp stay
// converged).  A key already there gets the value added; an empty slot is
// claimed with one CAS, and a CAS lost to another key re-reads the group
// from that slot, so slots are still taken in linear-probing order.
// Probing wraps from slot hi back to slot lo ([lo, hi) is the whole table,
// or a region whose bounds are multiples of 4).  Returns 0 when the probe
// limit is hit, 1 when the key existed, 2 when this call created it.
__device__ __forceinline__ int hash_add_from(unsigned long long* __restrict__ keys,
                                             long long* __restrict__ vals, uint64_t lo,
                                             uint64_t hi, uint64_t slot, uint32_t max_probe,
                                             unsigned long long key, long long v) {
  uint32_t probes = 0;
  while (probes < max_probe) {
    const uint64_t g = slot & ~3ull;
    // Slots of the group at or past hi (a table size that is not a multiple
    // of 4) are skipped; probing wraps to slot lo after the group.
    const uint32_t valid = (g + 4 <= hi) ? 4u : (uint32_t)(hi - g);
    unsigned long long k4[4];
    if (valid == 4) {
      // L2 loads: keys only ever change from EMPTY to a key, and a stale
      // EMPTY is caught by the CAS.
      const ulonglong2 a = __ldcg((const ulonglong2*)(keys + g));
      const ulonglong2 b = __ldcg((const ulonglong2*)(keys + g + 2));
      k4[0] = a.x; k4[1] = a.y; k4[2] = b.x; k4[3] = b.y;
    } else {
#pragma unroll
      for (uint32_t q = 0; q < 4; ++q) k4[q] = (q < valid) ? __ldcg(keys + g + q) : 0ull;
    }
    const uint32_t start = (uint32_t)(slot - g);
    uint32_t pick = 4;
#pragma unroll
    for (int q = 3; q >= 0; --q) {
      const bool usable = (uint32_t)q >= start && (uint32_t)q < valid &&
                          (k4[q] == key || k4[q] == EMPTY_KEY);
      pick = usable ? (uint32_t)q : pick;
    }
    if (pick == 4) {
      probes += valid > start ? valid - start : 0u;
      slot = g + 4;
      if (slot >= hi) slot = lo;
      continue;
    }
    probes += pick - start + 1;
    unsigned long long cur = k4[0];
#pragma unroll
    for (uint32_t q = 1; q < 4; ++q) cur = (q == pick) ? k4[q] : cur;
    int created = 0;
    if (cur != key) {
      const unsigned long long prev = atomicCAS(keys + g + pick, EMPTY_KEY, key);
      if (prev != EMPTY_KEY && prev != key) {
        slot = g + pick;  // taken by another key: look again from here
        continue;
      }
      created = prev == EMPTY_KEY ? 2 : 0;
    }
    atomicAdd((unsigned long long*)vals + g + pick, (unsigned long long)v);
    return created ? 2 : 1;
  }
  return 0;
}

// Log buckets of positive 64-bit values: 16 * floor(log2 v) + the 4 bits
// below the leading bit (1024 buckets, monotone in v), and a bucket's
// smallest value.
__device__ __forceinline__ uint32_t log_bucket(unsigned long long v) {
  const int e = 63 - __clzll((long long)v);
  const uint32_t f = e >= 4 ? (uint32_t)(v >> (e - 4)) & 15u : (uint32_t)(v << (4 - e)) & 15u;
  return (uint32_t)e * 16u + f;
}

__host__ __device__ __forceinline__ unsigned long long bucket_floor(uint32_t b) {
  const int e = (int)(b >> 4);
  const unsigned long long m = 16ull + (b & 15u);
  return e >= 4 ? (m << (e - 4)) : (m >> (4 - e));
}

// Bloom filter for the 0/1 closure test: a key sets five bits (five 6-bit
// fields of a second mix of its hash) in one 64-bit word (the top bits of
// its hash).  A clear bit proves the entry absent; a set filter sends the
// test to the exact search.
__device__ __forceinline__ unsigned long long bloom_bits(unsigned long long h) {
  const unsigned long long g = mix64(h ^ 0xA0761D6478BD642Full);
  return (1ull << (g & 63)) | (1ull << ((g >> 6) & 63)) | (1ull << ((g >> 12) & 63)) |
         (1ull << ((g >> 18) & 63)) | (1ull << ((g >> 24) & 63));
}

__device__ __forceinline__ bool bloom_may_contain(const unsigned long long* __restrict__ words,
                                                  int shift, unsigned long long key) {
  const unsigned long long h = mix64(key);
  const unsigned long long m = bloom_bits(h);
  return (__ldg(words + (h >> shift)) & m) == m;
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
  return hash_add_from(p.hkeys, p.hvals, 0, p.hcap, home_slot(p, key), p.max_probe, key, v);
}

// Histogram pick by one whole block of 256 threads: the highest bucket b
// whose count from the top (buckets b .. NB-1) reaches K, or -1 when the
// total stays below K; *total receives the sum of all buckets.  The counts
// are read from global memory (L2), each thread owning NB/256 consecutive
// buckets from the top, and a block scan finds the thread whose range the
// running count crosses.  Every thread of the block must call it.
template <int NB>
__device__ int block_pick_from_top(const unsigned int* hist, unsigned long long K,
                                   unsigned long long* total) {
  static_assert(NB % 256 == 0, "buckets per thread");
  constexpr int PER = NB / 256;
  __shared__ unsigned long long csum[256];
  __shared__ int pick;
  const int t = threadIdx.x;
  unsigned int v[PER];
  unsigned long long mine = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    v[q] = __ldcg(hist + (NB - 1 - (t * PER + q)));
    mine += v[q];
  }
  csum[t] = mine;
  if (t == 0) pick = -1;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    const unsigned long long add = t >= off ? csum[t - off] : 0ull;
    __syncthreads();
    csum[t] += add;
    __syncthreads();
  }
  const unsigned long long before = t ? csum[t - 1] : 0ull;
  if (before < K && csum[t] >= K) {
    unsigned long long cum = before;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      cum += v[q];
      if (cum >= K) {
        pick = NB - 1 - (t * PER + q);
        break;
      }
    }
  }
  __syncthreads();
  *total = csum[255];
  return pick;
}

}  // namespace mad
