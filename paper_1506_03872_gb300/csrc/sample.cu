// The sampling loop of Alg. 2: for every diamond index l, draw the center
// edge (i,k) with probability w_ik / ||W||_1 (two stages: row i from T1,
// then k from row i of T2), j with probability |b_kj| / ||b_k*||_1 (row k of
// TB), k' with probability |a_ik'| / ||a_i*||_1 (row i of TA), and add
// sgn(a_ik b_kj a_ik') b_k'j to x_ij (Alg. 2 increment line).
//
// GPU organisation: one diamond per thread; the signs of a_ik, b_kj and
// a_ik' come for free with the table entries the searches land on (bit 31),
// so only b_k'j is read from B.  Lanes of a warp whose diamonds hit the same
// key combine their increments before one lane inserts into the hash.
//
// Dense inputs are processed in row order: a counting sort by the row i of
// each diamond's center edge (drawn from T1 alone) groups the diamonds, so
// the lanes of a warp mostly share row i and its T2/TA/A entries come from
// L1 once per row instead of once per diamond, and the hash keys (i, j) of
// the rows in flight fall into a narrow band of home regions that stays in
// L2.  The draws of every diamond are unchanged by the reordering.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <type_traits>

#include "draw.cuh"
#include "mad_device.cuh"
#include "mad_internal.cuh"

namespace mad {
namespace {

// The scalars derived from T1's total on the device (and, for the dense
// hash, the end of its home regions), read once per thread, so that no
// host round trip separates the table build from the sampler.
__device__ __forceinline__ SampleParams resolve(const SampleParams& p) {
  SampleParams q = p;
  q.t1_total = p.sc->t1_total;
  q.t1g_sh = p.sc->t1g_sh;
  q.f_exp = p.sc->f_exp;
  if (p.regioned) {
    const unsigned long long used = p.hreg[p.m];
    q.hcap = used < p.hcap_alloc ? used : p.hcap_alloc;
  }
  return q;
}

// Per-lane bookkeeping of the sampling kernels.
struct Tally {
  unsigned long long inserted = 0, diag = 0, created = 0;
  bool bad = false, full = false;
};

// Filter one drawn diamond and add it to X.  Lanes holding the same key
// insert independently (the atomics combine them).
// One addition of v to the pair (a, b) (unordered under MAD_GRAM).
__device__ __forceinline__ void add_pair(const SampleParams& p, uint32_t a, uint32_t b, long long v,
                                         Tally& t) {
  if ((p.flags & MAD_EXCLUDE_DIAG) && a == b) {
    ++t.diag;
    return;
  }
  if (v == 0) return;
  if ((p.flags & MAD_GRAM) && b < a) {
    const uint32_t c = a;
    a = b;
    b = c;
  }
  ++t.inserted;
  const int r = hash_add(p, ((unsigned long long)a << 32) | b, v);
  if (r == 0) t.full = true;
  if (r == 2) ++t.created;
}

// Filter one drawn diamond and add it to X: to the pair (i, j), and under
// MAD_SQUARE_SYM also to the pair (k, k') (Sec. 3.2.3).  Lanes holding the
// same key insert independently (the atomics combine them).
__device__ __forceinline__ void accumulate(const SampleParams& p, bool valid, const Draw& dr,
                                           Tally& t) {
  if (!valid) return;
  add_pair(p, dr.i, dr.j, dr.v, t);
  if (p.flags & MAD_SQUARE_SYM) add_pair(p, dr.k, dr.kp, dr.v, t);
}

// The same, reduced over the whole block first (one atomic per counter and
// block: kernels with many short blocks would otherwise queue thousands of
// atomics on the same counters).  Every thread of the block calls it.
__device__ __forceinline__ void flush_tally_block(const SampleParams& p, Tally& t) {
  __shared__ unsigned long long s_ins, s_cre;
  __shared__ unsigned int s_flags;
  if (threadIdx.x == 0) {
    s_ins = 0;
    s_cre = 0;
    s_flags = 0;
  }
  __syncthreads();
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    t.inserted += __shfl_xor_sync(0xFFFFFFFFu, t.inserted, off);
    t.created += __shfl_xor_sync(0xFFFFFFFFu, t.created, off);
  }
  const unsigned any_full = __ballot_sync(0xFFFFFFFFu, t.full);
  if ((threadIdx.x & 31) == 0) {
    if (t.inserted) atomicAdd(&s_ins, t.inserted);
    if (t.created) atomicAdd(&s_cre, t.created);
    if (any_full) atomicOr(&s_flags, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_ins) atomicAdd(&p.sc->inserted, s_ins);
    if (s_cre) atomicAdd(&p.sc->new_keys, s_cre);
    if (s_flags) atomicOr(&p.sc->err, DERR_HASH_FULL);
  }
}

__device__ __forceinline__ void flush_tally(const SampleParams& p, Tally& t) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    t.inserted += __shfl_xor_sync(0xFFFFFFFFu, t.inserted, off);
    t.diag += __shfl_xor_sync(0xFFFFFFFFu, t.diag, off);
    t.created += __shfl_xor_sync(0xFFFFFFFFu, t.created, off);
  }
  const unsigned any_bad = __ballot_sync(0xFFFFFFFFu, t.bad);
  const unsigned any_full = __ballot_sync(0xFFFFFFFFu, t.full);
  if (lane == 0) {
    if (t.inserted) atomicAdd(&p.sc->inserted, t.inserted);
    if (t.diag) atomicAdd(&p.sc->diag_skipped, t.diag);
    if (t.created) atomicAdd(&p.sc->new_keys, t.created);
    if (any_bad) atomicOr(&p.sc->err, DERR_SEARCH);
    if (any_full) atomicOr(&p.sc->err, DERR_HASH_FULL);
  }
}

// Diamonds in index order (0/1 CSR inputs; dense inputs with alias draws).
template <bool kAlias>
__global__ void __launch_bounds__(256)
k_sample(const SampleParams p_, unsigned long long seed, unsigned long long first,
         unsigned long long s) {
  const SampleParams p = resolve(p_);
  const int lane = threadIdx.x & 31;
  const unsigned long long warp_id = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  Tally t;
  for (unsigned long long base = warp_id * 32; base < s; base += warps * 32) {
    const unsigned long long q = base + lane;
    Draw dr{};
    if (q < s) dr = draw_one_as<kAlias>(p, seed, first + q, &t.bad);
    accumulate(p, q < s, dr, t);
  }
  flush_tally(p, t);
}

// Counting sort of diamonds into row order.  A diamond's bucket is the top
// bits of its stage-1 target (Philox block 0 and T1's total only): the row
// i = upper_bound(T1, target) is non-decreasing in the target, so bucket
// order is row order; the T1 search itself is left to the draw kernel,
// where neighbouring diamonds search the same few lines of T1.  At most
// 2^kSortBitsMax buckets (a few rows each; measured on the dense factor
// workload, 2^14 buckets made sampling 3.7 % slower than 2^15).  One block
// per SM takes a contiguous chunk of the diamonds and counts them per
// bucket in shared memory (step 1), the counts become per-(bucket, block)
// offsets (steps 2 and 3), and each block places its diamonds by
// shared-memory counts (step 4): no global atomics and no per-diamond
// record between the steps.
constexpr int kSortBitsMax = 16;
// Above 2^15 buckets the shared-memory counters are 16 bits, two to a word:
// the buckets are equal slices of the uniform target range, each at most
// 2^-15 of it, so a block's chunk (at most 2^26 / #SMs diamonds) puts about
// 14 diamonds into a bucket, far below 2^16.
constexpr uint32_t kWideSort = 1u << 15;
// Row stride of the per-(block, bucket) counts: a power-of-two number of
// buckets plus 64 words, so that the rows of successive blocks do not all
// start on the same memory channel (the column passes read one entry of
// every row).
__host__ __device__ __forceinline__ size_t sort_row(uint32_t nbk) { return (size_t)nbk + 64; }

__device__ __forceinline__ uint32_t sort_bucket(unsigned long long ell, uint2 key,
                                                unsigned long long t1_total, int shift) {
  const uint4 b0 = philox4x32_10(make_uint4((uint32_t)ell, (uint32_t)(ell >> 32), 0u, 0u), key);
  const unsigned long long u0 = ((unsigned long long)b0.y << 32) | b0.x;
  return (uint32_t)(draw_target(u0, t1_total) >> shift);
}

// Step 1: H[g * sort_row(nbk) + b] = diamonds of block g's chunk in bucket b.
template <bool Packed>
__global__ void __launch_bounds__(1024)
k_sort_hist(const DevScalars* __restrict__ sc, unsigned long long seed, unsigned long long first,
            unsigned long long s, unsigned long long chunk, uint32_t nbk,
            unsigned int* __restrict__ H) {
  extern __shared__ unsigned int sort_cnt[];
  const uint32_t words = Packed ? nbk / 2 : nbk;
  for (uint32_t b = threadIdx.x; b < words; b += blockDim.x) sort_cnt[b] = 0;
  __syncthreads();
  const unsigned long long t1_total = sc->t1_total;
  const int shift = sc->sort_shift;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const unsigned long long q0 = (unsigned long long)blockIdx.x * chunk;
  const unsigned long long q1 = q0 + chunk < s ? q0 + chunk : s;
  for (unsigned long long q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    const uint32_t b = sort_bucket(first + q, key, t1_total, shift);
    if (Packed) atomicAdd(&sort_cnt[b >> 1], 1u << ((b & 1u) << 4));
    else atomicAdd(&sort_cnt[b], 1u);
  }
  __syncthreads();
  unsigned int* __restrict__ row = H + (size_t)blockIdx.x * sort_row(nbk);
  for (uint32_t b = threadIdx.x; b < nbk; b += blockDim.x)
    row[b] = Packed ? (sort_cnt[b >> 1] >> ((b & 1u) << 4)) & 0xFFFFu : sort_cnt[b];
}

// Step 2: tot[b] = sum over the blocks of H[g][b].
__global__ void __launch_bounds__(256)
k_sort_colsum(const unsigned int* __restrict__ H, uint32_t nbk, int blocks,
              unsigned int* __restrict__ tot) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbk) return;
  unsigned int acc = 0;
#pragma unroll 16
  for (int g = 0; g < blocks; ++g) acc += H[(size_t)g * sort_row(nbk) + b];
  tot[b] = acc;
}

// Step 3 (after the exclusive scan of tot into base): H[g][b] becomes the
// first position of block g's diamonds of bucket b.  Thirty-two loads are
// in flight before their stores (one thread walks all the blocks of its
// bucket; splitting the walk over more threads measured slower).
__global__ void __launch_bounds__(256)
k_sort_coloff(unsigned int* __restrict__ H, uint32_t nbk, int blocks,
              const unsigned int* __restrict__ base) {
  constexpr int kBatch = 32;
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbk) return;
  const size_t row = sort_row(nbk);
  unsigned int acc = base[b];
  int g = 0;
  for (; g + kBatch <= blocks; g += kBatch) {
    unsigned int c[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) c[u] = H[(size_t)(g + u) * row + b];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      H[(size_t)(g + u) * row + b] = acc;
      acc += c[u];
    }
  }
  for (; g < blocks; ++g) {
    const unsigned int c = H[(size_t)g * row + b];
    H[(size_t)g * row + b] = acc;
    acc += c;
  }
}

// Step 4: order[position] = q for every diamond q of the block's chunk.
// Unpacked: the block's offsets are staged as shared-memory cursors.
// Packed: a 16-bit shared-memory count gives the rank, added to the offset
// read from H.
template <bool Packed>
__global__ void __launch_bounds__(1024)
k_sort_scatter(const DevScalars* __restrict__ sc, unsigned long long seed,
               unsigned long long first, unsigned long long s, unsigned long long chunk,
               uint32_t nbk, const unsigned int* __restrict__ H, uint32_t* __restrict__ order) {
  extern __shared__ unsigned int sort_cnt[];
  const unsigned int* __restrict__ row = H + (size_t)blockIdx.x * sort_row(nbk);
  if (Packed) {
    for (uint32_t w = threadIdx.x; w < nbk / 2; w += blockDim.x) sort_cnt[w] = 0;
  } else {
    for (uint32_t b = threadIdx.x; b < nbk; b += blockDim.x) sort_cnt[b] = row[b];
  }
  __syncthreads();
  const unsigned long long t1_total = sc->t1_total;
  const int shift = sc->sort_shift;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const unsigned long long q0 = (unsigned long long)blockIdx.x * chunk;
  const unsigned long long q1 = q0 + chunk < s ? q0 + chunk : s;
  for (unsigned long long q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    const uint32_t b = sort_bucket(first + q, key, t1_total, shift);
    unsigned int pos;
    if (Packed) {
      const uint32_t sh = (b & 1u) << 4;
      pos = __ldg(row + b) + ((atomicAdd(&sort_cnt[b >> 1], 1u << sh) >> sh) & 0xFFFFu);
    } else {
      pos = atomicAdd(&sort_cnt[b], 1u);
    }
    order[pos] = (uint32_t)q;
  }
}

// Diamonds in row order (dense inputs): order[q] = l - first.  Draws only:
// diamond q's hash key goes to keys[q] (EMPTY_KEY when it adds nothing:
// v = 0 or an excluded diagonal) and its increment to vals[q].  Under
// MAD_SQUARE_SYM the same increment for the pair (k, k') goes to keys[s +
// q] and vals[s + q] (Sec. 3.2.3).  k_insert adds them to X.
__global__ void __launch_bounds__(256, 6)
k_sample_sorted(const SampleParams p_, unsigned long long seed, unsigned long long first,
                unsigned long long s, const uint32_t* __restrict__ order,
                unsigned long long* __restrict__ keys, long long* __restrict__ vals) {
  const bool sqsym = (p_.flags & MAD_SQUARE_SYM) != 0;
  const SampleParams p = resolve(p_);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  bool bad = false;
  unsigned long long diag = 0;
  for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < s;
       q += stride) {
    const Uniforms u = diamond_uniforms(seed, first + __ldcs(order + q));
    const int64_t i = draw_row_i(p, u.u0, &bad);
    const Draw dr = draw_given_row(p, u, i, &bad);
    unsigned long long key = EMPTY_KEY;
    if ((p.flags & MAD_EXCLUDE_DIAG) && dr.i == dr.j) {
      ++diag;
    } else if (dr.v != 0) {
      uint32_t a = dr.i, b = dr.j;
      if ((p.flags & MAD_GRAM) && b < a) {
        a = dr.j;
        b = dr.i;
      }
      key = ((unsigned long long)a << 32) | b;
    }
    keys[q] = key;
    vals[q] = dr.v;
    if (sqsym) {
      unsigned long long key2 = EMPTY_KEY;
      if ((p.flags & MAD_EXCLUDE_DIAG) && dr.k == dr.kp) {
        ++diag;
      } else if (dr.v != 0) {
        const uint32_t a = dr.k < dr.kp ? dr.k : dr.kp, b = dr.k < dr.kp ? dr.kp : dr.k;
        key2 = ((unsigned long long)a << 32) | b;
      }
      keys[s + q] = key2;
      vals[s + q] = dr.v;
    }
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) diag += __shfl_xor_sync(0xFFFFFFFFu, diag, off);
  const unsigned any_bad = __ballot_sync(0xFFFFFFFFu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (diag) atomicAdd(&p.sc->diag_skipped, diag);
    if (any_bad) atomicOr(&p.sc->err, DERR_SEARCH);
  }
}

// X update for the row-ordered diamonds: a lean kernel (full occupancy) so
// many inserts are in flight at once; consecutive entries share row i and
// hence its hash region.
__global__ void __launch_bounds__(256, 6)
k_insert(const SampleParams p_, const unsigned long long* __restrict__ keys,
         const long long* __restrict__ vals, unsigned long long s) {
  const SampleParams p = resolve(p_);
  Tally t;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long rounds = (s + stride - 1) / stride;
  // The next entry is loaded before the current one is inserted.
  unsigned long long key = q < s ? __ldcs(keys + q) : EMPTY_KEY;
  long long v = q < s ? __ldcs(vals + q) : 0;
  for (unsigned long long r = 0; r < rounds; ++r) {
    const unsigned long long qn = q + stride;
    const unsigned long long key_n = qn < s ? __ldcs(keys + qn) : EMPTY_KEY;
    const long long v_n = qn < s ? __ldcs(vals + qn) : 0;
    if (key != EMPTY_KEY) {
      ++t.inserted;
      const int res = hash_add(p, key, v);
      if (res == 0) t.full = true;
      if (res == 2) ++t.created;
    }
    key = key_n;
    v = v_n;
    q = qn;
  }
  flush_tally(p, t);
}

// (key, value) pairs added to X as k_insert adds drawn diamonds: partial X
// of other diamond ranges merged into this context's X (sharded runs).
// Counts the keys it creates, not diamonds.
__global__ void __launch_bounds__(256)
k_accumulate(const SampleParams p_, const unsigned long long* __restrict__ keys,
             const long long* __restrict__ vals, unsigned long long n) {
  const SampleParams p = resolve(p_);
  Tally t;
  for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long key = keys[q];
    if (key == EMPTY_KEY) continue;
    const int res = hash_add(p, key, vals[q]);
    if (res == 0) t.full = true;
    if (res == 2) ++t.created;
  }
  flush_tally(p, t);
}

// ---- X from empty, one group of rows per block -----------------------------
// When a single sorted batch of diamonds fills an empty X (the fused pass),
// the home regions are written whole instead of cleared and then updated
// with global atomics.  The sort buckets are taken 2^lg_group at a time; group
// g covers the targets [g << gs, (g + 1) << gs) with gs = sort shift +
// lg_group and owns the rows whose first target lies there,
// [R[g], R[g+1]) with R[0] = 0, R[g] = 1 + #{r : T1[r] < g << gs} and
// R[last + 1] = m.  Their regions, [hreg[R[g]], hreg[R[g+1]]), are
// contiguous.  A block builds them in shared memory from the diamonds of its
// buckets (those of its last row that fall into later buckets included) and
// stores them with plain coalesced writes, so X is written once and never read
// back from DRAM.  Every key probes linearly from its home slot through its
// group's regions, taken as one circular table; a key that finds them all
// full goes to the overflow table after the regions, [hreg[m], hreg[m] + O),
// a plain linear-probing hash.  Groups whose regions exceed the
// shared-memory image are "heavy": a first kernel clears their regions and
// the diamonds of their rows are added with global atomics (the same
// circular probing) by whichever block holds them in its own buckets.
// Each diamond is added exactly once, so X is the same set of
// (key, sum) as the one k_insert builds (the sums are exact integers).
constexpr int kImageSlots = 3072;   // 48 KB: keys, then values
constexpr int kRowCache = 256;      // owned rows whose hreg a block keeps in shared memory

// R[h] for a group boundary h (see above): 1 + #{r : T1[r] < h << gs}, read
// from the T1 guide (entry b counts the T1 entries below b << t1g_sh, and
// gs >= t1g_sh: the boundary is on a guide bucket).
__device__ __forceinline__ int64_t group_first_row(const SampleParams& p, uint32_t h,
                                                   uint32_t ngroups, int gs) {
  if (h == 0) return 0;
  if (h >= ngroups) return p.m;
  const unsigned long long t = (unsigned long long)h << gs;
  if (t > p.t1_total) return p.m;
  const int64_t r = (int64_t)__ldg(p.T1g + (t >> p.t1g_sh)) + 1;
  return r < p.m ? r : p.m;
}

// Row bounds of every group (R), its heavy flag, the sorted position where
// the diamonds it builds end (qend: its own buckets and those of its last
// row's diamonds), the clearing of heavy groups' regions and of the
// overflow table.  One warp per group.
__global__ void __launch_bounds__(256)
k_group_prep(const SampleParams p_, const unsigned int* __restrict__ base, uint32_t nbk,
             int lg_group, uint32_t ngroups, uint64_t ov_slots, int narrow,
             uint32_t* __restrict__ R, unsigned char* __restrict__ heavy,
             uint32_t* __restrict__ qend) {
  const SampleParams p = resolve(p_);
  const int lane = threadIdx.x & 31;
  const uint32_t g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int gs = p.sc->sort_shift + lg_group;
  const unsigned long long ov0 = p.hreg[p.m];
  if (ov0 + ov_slots > p.hcap_alloc) {   // (the allocation bounds the regions)
    if (g == 0 && lane == 0) atomicOr(&p.sc->err, DERR_HASH_FULL);
    return;
  }
  if (g < ngroups) {
    unsigned long long slot = 0, tend = 0;
    int64_t r = 0;
    if (lane < 2) {
      r = group_first_row(p, g + lane, ngroups, gs);
      slot = p.hreg[r];
      if (lane == 1 && r > 0) tend = p.T1[r - 1];   // where the last owned row's targets end
      if (lane == 0) R[g] = (uint32_t)r;
      if (lane == 1 && g + 1 == ngroups) R[ngroups] = (uint32_t)p.m;
    }
    const unsigned long long lo = __shfl_sync(0xFFFFFFFFu, slot, 0);
    const unsigned long long hi = __shfl_sync(0xFFFFFFFFu, slot, 1);
    const int64_t r0 = __shfl_sync(0xFFFFFFFFu, r, 0);
    const int64_t r1 = __shfl_sync(0xFFFFFFFFu, r, 1);
    // Narrow image keys name the row by its offset in the group (8 bits).
    const bool big = hi - lo > (unsigned long long)kImageSlots ||
                     (narrow && r1 - r0 >= (int64_t)kRowCache);
    if (lane == 1) {
      // The sorted position where the diamonds the group builds end: its
      // own buckets, and those of its last row.
      const int bsh = p.sc->sort_shift;
      const uint32_t b1 = (g + 1) << lg_group;
      unsigned long long be = (tend >> bsh) + ((tend & ((1ull << bsh) - 1)) ? 1 : 0);
      be = be < nbk ? be : nbk;
      qend[g] = (!big && r > r0 && be > b1) ? base[be] : base[b1];
    }
    if (lane == 0) heavy[g] = big ? 1 : 0;
    if (big)
      for (unsigned long long x = lo + lane; x < hi; x += 32) {
        p.hkeys[x] = EMPTY_KEY;
        p.hvals[x] = 0;
      }
  }
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       x < ov_slots; x += (unsigned long long)gridDim.x * blockDim.x) {
    p.hkeys[ov0 + x] = EMPTY_KEY;
    p.hvals[ov0 + x] = 0;
  }
}

// Global insert of key into the circular table [lo, hi) from slot, then,
// when it is full, into the overflow table.  1 existing key, 2 new key, 0
// both full.
__device__ __forceinline__ int add_span_or_overflow(const SampleParams& p, unsigned long long lo,
                                                    unsigned long long hi, unsigned long long slot,
                                                    unsigned long long ov0, uint64_t ov_slots,
                                                    unsigned long long key, long long v) {
  if (lo < hi) {
    const int r = hash_add_from(p.hkeys, p.hvals, lo, hi, slot, (uint32_t)(hi - lo), key, v);
    if (r) return r;
  }
  return hash_add_from(p.hkeys, p.hvals, ov0, ov0 + ov_slots, ov0 + (mix64(key) & (ov_slots - 1)),
                       (uint32_t)ov_slots, key, v);
}

// The regions of group blockIdx.x (see above).  base[b] is the first sorted
// position of bucket b (base[nbk] = the batch size); R, heavy and qend_g
// come from k_group_prep.
//
// kNarrow: the image holds 32-bit keys, (row - first owned row) << 24 | j,
// for n <= 2^24 and groups of fewer than kRowCache rows (k_group_prep makes
// larger groups heavy): the key claim is a 32-bit compare-and-swap and one
// 16-byte shared load reads four probe slots.  Otherwise the image holds
// the 64-bit keys.  The stored X holds 64-bit keys either way.
template <bool kNarrow>
__global__ void __launch_bounds__(256)
k_build_x(const SampleParams p_, const unsigned long long* __restrict__ keys,
          const long long* __restrict__ vals, const unsigned int* __restrict__ base,
          uint32_t nbk, int lg_group, uint32_t ngroups, uint64_t ov_slots,
          const uint32_t* __restrict__ R, const unsigned char* __restrict__ heavy,
          const uint32_t* __restrict__ qend_g) {
  // kImageSlots keys (4 or 8 bytes), then kImageSlots 8-byte values.
  extern __shared__ __align__(16) unsigned long long img[];
  using IKey = typename std::conditional<kNarrow, uint32_t, unsigned long long>::type;
  constexpr IKey kEmptyI = (IKey)~(IKey)0;
  __shared__ uint32_t s_off[kRowCache + 1];   // owned rows' region offsets in the image
  const SampleParams p = resolve(p_);
  const unsigned long long ov0 = p.hreg[p.m];
  if (ov0 + ov_slots > p.hcap_alloc) return;   // reported by k_group_prep
  const uint32_t g = blockIdx.x;
  const int bsh = p.sc->sort_shift;
  const int gs = bsh + lg_group;
  const uint32_t b0 = g << lg_group;
  const uint32_t b1 = b0 + (1u << lg_group) < nbk ? b0 + (1u << lg_group) : nbk;
  // Every thread reads the group's bounds (one broadcast round trip), then
  // its regions' bounds and its first diamond.
  const uint32_t r0 = R[g], r1 = R[g + 1];
  const unsigned long long q0 = base[b0], q1 = base[b1], qend = qend_g[g];
  const bool hv = heavy[g] != 0;
  const unsigned long long lo = p.hreg[r0];
  const unsigned long long span = hv ? 0 : p.hreg[r1] - lo;
  const bool cached = r1 - r0 < (uint32_t)kRowCache;
  if (!hv && cached)
    for (uint32_t x = threadIdx.x; x <= r1 - r0; x += blockDim.x)
      s_off[x] = (uint32_t)(p.hreg[r0 + x] - lo);
  const uint32_t span32 = (uint32_t)span;
  unsigned long long q = q0 + threadIdx.x;
  unsigned long long key = q < qend ? keys[q] : EMPTY_KEY;
  long long v = q < qend ? vals[q] : 0;
  IKey* ik = (IKey*)img;
  unsigned long long* iv = (unsigned long long*)((char*)img + kImageSlots * sizeof(IKey));
  for (uint32_t x = 4 * threadIdx.x; x < span32; x += 4 * blockDim.x) {
    if (kNarrow) {
      *(uint4*)(ik + x) = make_uint4(~0u, ~0u, ~0u, ~0u);
    } else {
      *(ulonglong2*)(ik + x) = make_ulonglong2(EMPTY_KEY, EMPTY_KEY);
      *(ulonglong2*)(ik + x + 2) = make_ulonglong2(EMPTY_KEY, EMPTY_KEY);
    }
    *(ulonglong2*)(iv + x) = make_ulonglong2(0, 0);
    *(ulonglong2*)(iv + x + 2) = make_ulonglong2(0, 0);
  }
  __syncthreads();
  Tally t;
  for (; q < qend; q += blockDim.x) {
    // The next diamond is loaded before this one is added.
    const unsigned long long qn = q + blockDim.x;
    const unsigned long long key_n = qn < qend ? keys[qn] : EMPTY_KEY;
    const long long v_n = qn < qend ? vals[qn] : 0;
    const unsigned long long k = key;
    const long long w = v;
    key = key_n;
    v = v_n;
    if (k == EMPTY_KEY) continue;
    const uint32_t i = (uint32_t)(k >> 32);
    const bool own = !hv && i >= r0 && i < r1;
    int res;
    if (own) {
      // Linear probe of the image from the home slot, wrapping at its end
      // (the group's regions form one circular table), four slots per
      // step (two 16-byte shared loads; regions start on 4-slot groups).
      // A stale EMPTY is caught by the CAS; a key once set never changes.
      // Image positions are 32-bit (the image holds kImageSlots slots).
      uint32_t roff, rsz;
      if (cached) {
        roff = s_off[i - r0];
        rsz = s_off[i - r0 + 1] - roff;
      } else {
        const unsigned long long a = __ldg(p.hreg + i);
        roff = (uint32_t)(a - lo);
        rsz = (uint32_t)(__ldg(p.hreg + i + 1) - a);
      }
      uint32_t x = roff + (fmix32((uint32_t)k) & (rsz - 1));
      const IKey kk = kNarrow ? (IKey)(((i - r0) << 24) | (uint32_t)k) : (IKey)k;
      res = 0;
      for (uint32_t probes = 0; probes < span32;) {
        const uint32_t gx = x & ~3u;
        IKey k4[4];
        if (kNarrow) {
          const uint4 ka = *(const uint4*)(ik + gx);
          k4[0] = (IKey)ka.x; k4[1] = (IKey)ka.y; k4[2] = (IKey)ka.z; k4[3] = (IKey)ka.w;
        } else {
          const ulonglong2 ka = *(const ulonglong2*)(ik + gx);
          const ulonglong2 kb = *(const ulonglong2*)(ik + gx + 2);
          k4[0] = (IKey)ka.x; k4[1] = (IKey)ka.y; k4[2] = (IKey)kb.x; k4[3] = (IKey)kb.y;
        }
        const uint32_t start = x - gx;
        uint32_t pick = 4;
#pragma unroll
        for (int u = 3; u >= 0; --u)
          pick = ((uint32_t)u >= start && (k4[u] == kk || k4[u] == kEmptyI)) ? (uint32_t)u : pick;
        if (pick == 4) {
          probes += 4 - start;
          x = gx + 4 < span32 ? gx + 4 : 0;
          continue;
        }
        probes += pick - start + 1;
        IKey cur = k4[0];
#pragma unroll
        for (int u = 1; u < 4; ++u) cur = (uint32_t)u == pick ? k4[u] : cur;
        const uint32_t slot = gx + pick;
        const IKey prev = cur == kk ? kk : atomicCAS(ik + slot, kEmptyI, kk);
        if (prev == kEmptyI || prev == kk) {
          // The 64-bit sum as two 32-bit shared atomics: the low word's own
          // carry goes into the high word, so the total is the exact sum.
          unsigned int* h2 = (unsigned int*)(iv + slot);
          const unsigned int wlo = (unsigned int)w;
          const unsigned int whi = (unsigned int)((unsigned long long)w >> 32);
          const unsigned int olo = atomicAdd(h2, wlo);
          atomicAdd(h2 + 1, whi + (olo + wlo < olo ? 1u : 0u));
          res = prev == kEmptyI ? 2 : 1;
          break;
        }
        x = slot + 1 < span32 ? slot + 1 : 0;   // taken by another key: go on after it
      }
      if (res == 0) res = add_span_or_overflow(p, 0, 0, 0, ov0, ov_slots, k, w);
    } else {
      if (q >= q1) continue;   // the owner's extension: not this block's
      const unsigned long long ex = i ? __ldg(p.T1 + i - 1) : 0ull;
      unsigned long long og = ex >> gs;
      og = og < ngroups - 1 ? og : ngroups - 1;
      if (!heavy[og]) continue;   // its owner builds it
      const unsigned long long rlo = __ldg(p.hreg + i), rhi = __ldg(p.hreg + i + 1);
      const unsigned long long home = rlo + (fmix32((uint32_t)k) & (rhi - rlo - 1));
      res = add_span_or_overflow(p, p.hreg[R[og]], p.hreg[R[og + 1]], home, ov0, ov_slots, k, w);
    }
    ++t.inserted;
    if (res == 0) t.full = true;
    if (res == 2) ++t.created;
  }
  __syncthreads();
  // The image, 16 bytes per store (regions start on 4-slot groups), keys
  // widened back to (i << 32) | j.
  for (uint32_t x = 2 * threadIdx.x; x < span32; x += 2 * blockDim.x) {
    unsigned long long k0, k1;
    if (kNarrow) {
      const uint32_t a = ik[x], b = ik[x + 1];
      k0 = a == ~0u ? EMPTY_KEY
                    : ((unsigned long long)(r0 + (a >> 24)) << 32) | (a & 0xFFFFFFu);
      k1 = b == ~0u ? EMPTY_KEY
                    : ((unsigned long long)(r0 + (b >> 24)) << 32) | (b & 0xFFFFFFu);
    } else {
      k0 = (unsigned long long)ik[x];
      k1 = (unsigned long long)ik[x + 1];
    }
    *(ulonglong2*)(p.hkeys + lo + x) = make_ulonglong2(k0, k1);
    *(longlong2*)(p.hvals + lo + x) = make_longlong2((long long)iv[x], (long long)iv[x + 1]);
  }
  flush_tally_block(p, t);
}

// Diagnostic twin of k_sample: writes each diamond's draws instead of
// accumulating them.
__global__ void __launch_bounds__(256)
k_draws(const SampleParams p_, unsigned long long seed, unsigned long long first,
        const unsigned long long* __restrict__ ells, unsigned long long count, uint32_t* oi,
        uint32_t* ok, uint32_t* oj, uint32_t* okp, long long* ov) {
  const SampleParams p = resolve(p_);
  bool bad = false;
  for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long ell = ells ? ells[q] : first + q;
    const Draw dr = draw_one(p, seed, ell, &bad);
    oi[q] = dr.i;
    ok[q] = dr.k;
    oj[q] = dr.j;
    okp[q] = dr.kp;
    ov[q] = dr.v;
  }
  if (bad) atomicOr(&p.sc->err, DERR_SEARCH);
}

// Resident 256-thread blocks of `kernel` on the whole GPU (queried once
// per kernel; one process drives one device).
template <auto kernel>
int full_grid() {
  static int cached = 0;
  if (cached) return cached;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  cached = sms * per_sm;
  return cached;
}

unsigned grid_of(unsigned long long work, int full) {
  const unsigned long long need = (work + 255) / 256;
  return (unsigned)(need < (unsigned long long)full ? (need ? need : 1) : full);
}

// Diamonds per sorted batch (bounds the scratch at 20 bytes per diamond).
constexpr unsigned long long kSortBatch = 1ull << 26;

// Pilot for hash sizing: counts the diamonds that would be inserted.
__global__ void __launch_bounds__(256)
k_pilot(const SampleParams p_, unsigned long long seed, unsigned long long n,
        unsigned long long* __restrict__ hits) {
  const SampleParams p = resolve(p_);
  bool bad = false;
  unsigned long long c = 0;
  for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (unsigned long long)gridDim.x * blockDim.x) {
    const Draw dr = draw_one_as<false>(p, seed, q, &bad);
    c += (dr.v != 0 && !((p.flags & MAD_EXCLUDE_DIAG) && dr.i == dr.j)) ? 1 : 0;
    if (p.flags & MAD_SQUARE_SYM)
      c += (dr.v != 0 && !((p.flags & MAD_EXCLUDE_DIAG) && dr.k == dr.kp)) ? 1 : 0;
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(hits, c);
  if (bad) atomicOr(&p.sc->err, DERR_SEARCH);
}

// Caller's profiling event q (if set) on the sampling stream.
void phase_event(const mad_ctx* ctx, uint32_t q, cudaStream_t st) {
  if (q < ctx->n_phase_ev && ctx->phase_ev[q]) cudaEventRecord(ctx->phase_ev[q], st);
}

}  // namespace

SampleParams make_params(const mad_ctx* ctx) {
  SampleParams p;
  p.a_val = ctx->A.values;
  p.a_ptr = ctx->A.rowptr;
  p.a_col = ctx->A.colidx;
  p.m = ctx->m;
  p.d = ctx->d;
  p.lda = ctx->A.ld;
  p.b_val = ctx->B.values;
  p.b_ptr = ctx->B.rowptr;
  p.b_col = ctx->B.colidx;
  p.n = ctx->n;
  p.ldb = ctx->B.ld;
  p.T1 = ctx->T1;
  p.T2 = ctx->T2;
  p.TA = ctx->TA;
  p.TB = ctx->TB;
  p.t1_total = ctx->t1_total;
  p.T1g = ctx->T1g;
  p.t1g_sh = ctx->t1g_sh;
  p.T2g_ptr = ctx->T2g_ptr;
  p.T2g = ctx->T2g;
  p.T2g_sh = ctx->T2g_sh;
  p.bloom = ctx->bloom;
  p.bloom_shift = 64 - ctx->bloom_lg;
  p.TBg = ctx->TBg;
  p.tbg_stride = ctx->tbg_stride;
  p.TBg_sh = ctx->TBg_sh;
  p.f_exp = ctx->f;
  p.hkeys = ctx->hkeys;
  p.hvals = ctx->hvals;
  p.hreg = ctx->hreg;
  p.hmask = ctx->hcap - 1;
  p.hcap = ctx->hcap;
  p.hcap_alloc = ctx->hcap_alloc;
  p.max_probe = (uint32_t)(ctx->hcap < 4096 ? ctx->hcap : 4096);
  p.regioned = ctx->regioned ? 1 : 0;
  p.dense = ctx->dense ? 1 : 0;
  p.a_f64 = ctx->A.dt == MAD_F64;
  p.b_f64 = ctx->B.dt == MAD_F64;
  p.integer = ctx->integer ? 1 : 0;
  p.flags = ctx->flags;
  p.sc = ctx->sc;
  p.alias = (ctx->flags & MAD_ALIAS) && ctx->al[kAlT1] ? 1 : 0;
  for (int f = 0; f < 4; ++f) {
    p.al[f] = ctx->al[f];
    p.al_seg[f] = ctx->al_seg[f];
    p.al_row[f] = ctx->al_row[f];
    p.al_nseg[f] = ctx->al_nseg[f];
  }
  return p;
}

mad_status pilot_inserts(mad_ctx* ctx, uint64_t n, uint64_t* hits, cudaStream_t st) {
  mad_status rs = ensure_scratch(ctx, 256, st);
  if (rs != MAD_OK) return rs;
  unsigned long long* dev = (unsigned long long*)ctx->scratch;
  cudaMemsetAsync(dev, 0, sizeof(unsigned long long), st);
  const SampleParams p = make_params(ctx);
  k_pilot<<<grid_of(n, full_grid<k_pilot>()), 256, 0, st>>>(p, 0x9E3779B97F4A7C15ull, n, dev);
  count_launch(ctx);
  unsigned long long h = 0;
  cudaMemcpyAsync(&h, dev, sizeof(h), cudaMemcpyDeviceToHost, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  *hits = h;
  return MAD_OK;
}

int sort_bits(int64_t m) {
  int lg = 0;
  while (lg < kSortBitsMax && (1ll << lg) < m) ++lg;
  return lg;
}

uint64_t sort_buckets(int64_t m) { return 1ull << sort_bits(m); }

// Blocks of the sort (one per SM).
int sort_blocks() {
  static int blocks = 0;
  if (!blocks) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&blocks, cudaDevAttrMultiProcessorCount, dev);
    if (blocks < 1) blocks = 1;
  }
  return blocks;
}

// Scratch of the sort and the draws for one batch: the per-(block, bucket)
// counts, bucket totals and offsets, the scan's partials, the diamond
// indices in bucket order, and each diamond's key and increment.
struct SortScratch {
  unsigned int* H;
  unsigned int* tot;
  unsigned int* base;
  unsigned int* part;
  uint32_t* order;
  unsigned long long* keys;
  long long* vals;
  uint32_t* R;              // row bounds of the X builder's groups
  unsigned char* heavy;     // their heavy flags
  uint32_t* qend;           // where the diamonds each group builds end
  size_t bytes;
};

// recs: records per diamond (2 under MAD_SQUARE_SYM).
SortScratch carve_sort(void* p, uint64_t nbk, int blocks, uint64_t batch, int recs) {
  SortScratch c;
  char* b = (char*)p;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = b ? b + off : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return (void*)q;
  };
  c.H = (unsigned int*)take(sort_row((uint32_t)nbk) * blocks * sizeof(unsigned int));
  c.tot = (unsigned int*)take(nbk * sizeof(unsigned int));
  c.base = (unsigned int*)take((nbk + 1) * sizeof(unsigned int));
  c.part = (unsigned int*)take(scan_partial_elems(nbk) * sizeof(unsigned int));
  c.order = (uint32_t*)take(batch * sizeof(uint32_t));
  c.keys = (unsigned long long*)take(batch * recs * sizeof(unsigned long long));
  c.vals = (long long*)take(batch * recs * sizeof(long long));
  c.R = (uint32_t*)take((nbk + 1) * sizeof(uint32_t));
  c.heavy = (unsigned char*)take(nbk);
  c.qend = (uint32_t*)take(nbk * sizeof(uint32_t));
  c.bytes = off;
  return c;
}

int sort_records(const mad_ctx* ctx) { return (ctx->flags & MAD_SQUARE_SYM) ? 2 : 1; }

size_t sample_scratch_bytes(const mad_ctx* ctx, uint64_t s) {
  if (!ctx->dense || s == 0) return 0;
  const uint64_t batch = s < kSortBatch ? s : kSortBatch;
  return carve_sort(nullptr, sort_buckets(ctx->m), sort_blocks(), batch, sort_records(ctx)).bytes;
}

// Buckets per group of the X builder: about 640 diamonds of s_max per group
// (regions of about 1300 slots against the 3072-slot image).
int build_group_log2(uint64_t nbk, uint64_t s_max) {
  int lg = 0;
  while ((2ull << lg) <= nbk && (2ull << lg) * s_max <= 640ull * nbk) ++lg;
  return lg;
}

bool x_builder_applies(const mad_ctx* ctx, uint64_t s) {
  return ctx->dense && ctx->regioned && ctx->hov > 0 && s > 0 && s <= kSortBatch &&
         !(ctx->flags & MAD_GRAM);
}

mad_status sample_impl(mad_ctx* ctx, uint64_t s, uint64_t seed, uint64_t first, cudaStream_t st,
                       bool fresh_x) {
  if (s == 0) return MAD_OK;
  if (ctx->flags & MAD_WEDGE) return wedge_sample_impl(ctx, s, seed, first, st);
  const SampleParams p = make_params(ctx);
  // 0/1 inputs, and alias draws (their row is not monotone in the uniform,
  // so the row-order sort does not apply): diamonds in index order.
  if (!ctx->dense || p.alias) {
    phase_event(ctx, 0, st);
    phase_event(ctx, 1, st);
    if (p.alias)
      k_sample<true><<<grid_of(s, full_grid<k_sample<true>>()), 256, 0, st>>>(p, seed, first, s);
    else
      k_sample<false><<<grid_of(s, full_grid<k_sample<false>>()), 256, 0, st>>>(p, seed, first, s);
    count_launch(ctx);
    phase_event(ctx, 2, st);
    phase_event(ctx, 3, st);
    return cuda_status(cudaGetLastError());
  }
  const int full_sorted = full_grid<k_sample_sorted>();
  const int full_insert = full_grid<k_insert>();
  const uint64_t nbk = sort_buckets(ctx->m);
  const int blocks = sort_blocks();
  const bool packed = nbk > kWideSort;
  const size_t sort_smem = (packed ? nbk / 2 : nbk) * sizeof(unsigned int);
  static size_t smem_set = 0;
  if (sort_smem > 48 * 1024 && smem_set < sort_smem) {
    cudaFuncSetAttribute(k_sort_hist<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sort_smem);
    cudaFuncSetAttribute(k_sort_hist<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sort_smem);
    cudaFuncSetAttribute(k_sort_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sort_smem);
    cudaFuncSetAttribute(k_sort_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sort_smem);
    smem_set = sort_smem;
  }
  const uint64_t batch = s < kSortBatch ? s : kSortBatch;
  // An empty X filled by one batch, keys owned by their drawn row: the
  // regions are built whole (k_build_x); otherwise k_insert adds to X.
  const bool build_x = fresh_x && x_builder_applies(ctx, s);
  // Narrow image keys when every column index fits in 24 bits.
  const bool narrow = ctx->n <= (1ll << 24);
  const size_t image_smem =
      (size_t)kImageSlots * ((narrow ? sizeof(uint32_t) : sizeof(unsigned long long)) +
                             sizeof(unsigned long long));
  static bool image_attr = false;
  if (build_x && !image_attr) {
    const int wide_smem = (int)(2 * (size_t)kImageSlots * sizeof(unsigned long long));
    cudaFuncSetAttribute(k_build_x<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, wide_smem);
    cudaFuncSetAttribute(k_build_x<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, wide_smem);
    image_attr = true;
  }
  mad_status rs = ensure_scratch(ctx, sample_scratch_bytes(ctx, s), st);
  if (rs != MAD_OK) return rs;
  const SortScratch w = carve_sort(ctx->scratch, nbk, blocks, batch, sort_records(ctx));
  for (uint64_t done = 0; done < s; done += batch) {
    const uint64_t n = (s - done) < batch ? (s - done) : batch;
    phase_event(ctx, 0, st);
    const unsigned long long chunk = (n + blocks - 1) / blocks;
    const unsigned cols = (unsigned)((nbk + 255) / 256);
    if (packed)
      k_sort_hist<true><<<blocks, 1024, sort_smem, st>>>(ctx->sc, seed, first + done, n, chunk,
                                                         (uint32_t)nbk, w.H);
    else
      k_sort_hist<false><<<blocks, 1024, sort_smem, st>>>(ctx->sc, seed, first + done, n, chunk,
                                                          (uint32_t)nbk, w.H);
    k_sort_colsum<<<cols, 256, 0, st>>>(w.H, (uint32_t)nbk, blocks, w.tot);
    if ((rs = scan_exclusive_u32(ctx, w.tot, w.base, nbk, w.part, st)) != MAD_OK) return rs;
    k_sort_coloff<<<cols, 256, 0, st>>>(w.H, (uint32_t)nbk, blocks, w.base);
    if (packed)
      k_sort_scatter<true><<<blocks, 1024, sort_smem, st>>>(ctx->sc, seed, first + done, n, chunk,
                                                            (uint32_t)nbk, w.H, w.order);
    else
      k_sort_scatter<false><<<blocks, 1024, sort_smem, st>>>(ctx->sc, seed, first + done, n,
                                                             chunk, (uint32_t)nbk, w.H, w.order);
    count_launch(ctx, 4);
    phase_event(ctx, 1, st);
    k_sample_sorted<<<grid_of(n, full_sorted), 256, 0, st>>>(p, seed, first + done, n, w.order,
                                                             w.keys, w.vals);
    count_launch(ctx);
    phase_event(ctx, 2, st);
    if (build_x) {
      const int lg = build_group_log2(nbk, ctx->s_max);
      const uint32_t ngroups = (uint32_t)(nbk >> lg);
      k_group_prep<<<(ngroups + 7) / 8, 256, 0, st>>>(p, w.base, (uint32_t)nbk, lg, ngroups,
                                                      ctx->hov, narrow ? 1 : 0, w.R, w.heavy,
                                                      w.qend);
      if (narrow)
        k_build_x<true><<<ngroups, 256, image_smem, st>>>(p, w.keys, w.vals, w.base,
                                                          (uint32_t)nbk, lg, ngroups, ctx->hov,
                                                          w.R, w.heavy, w.qend);
      else
        k_build_x<false><<<ngroups, 256, image_smem, st>>>(p, w.keys, w.vals, w.base,
                                                           (uint32_t)nbk, lg, ngroups, ctx->hov,
                                                           w.R, w.heavy, w.qend);
      count_launch(ctx, 2);
    } else {
      k_insert<<<grid_of(n, full_insert), 256, 0, st>>>(p, w.keys, w.vals,
                                                        n * (uint64_t)sort_records(ctx));
      count_launch(ctx);
    }
    phase_event(ctx, 3, st);
  }
  return cuda_status(cudaGetLastError());
}

mad_status accumulate_pairs(mad_ctx* ctx, const uint64_t* keys, const int64_t* vals, uint64_t n,
                            cudaStream_t st) {
  if (n == 0) return MAD_OK;
  const SampleParams p = make_params(ctx);
  k_accumulate<<<grid_of(n, full_grid<k_accumulate>()), 256, 0, st>>>(
      p, (const unsigned long long*)keys, (const long long*)vals, n);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

mad_status debug_draws_impl(mad_ctx* ctx, uint64_t seed, uint64_t first, const uint64_t* ells,
                            uint64_t count, uint32_t* oi, uint32_t* ok, uint32_t* oj,
                            uint32_t* okp, int64_t* ov, cudaStream_t st) {
  if (count == 0) return MAD_OK;
  if (ctx->flags & MAD_WEDGE)
    return wedge_draws_impl(ctx, seed, first, ells, count, oi, ok, oj, okp, ov, st);
  const SampleParams p = make_params(ctx);
  const unsigned long long blocks = (count + 255) / 256;
  k_draws<<<(unsigned)(blocks < 152 * 8 ? blocks : 152 * 8), 256, 0, st>>>(
      p, seed, first, (const unsigned long long*)ells, count, oi, ok, oj, okp, (long long*)ov);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

}  // namespace mad
