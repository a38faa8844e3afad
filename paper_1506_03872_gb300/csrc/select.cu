// Top-K selection for Alg. 3: Omega_t' (the t' largest x_ij) and Omega_t
// (the t largest |c_ij|).  Items carry a primary key p (larger first) and a
// tie key (smaller first); since keys are distinct, the composite
// (p, ~key) orders items totally and the K-th largest composite is unique.
//
// 1. Hash path: one pass builds a 1024-bucket logarithmic histogram of the
//    positive x; the bucket where the count from the top reaches K gives a
//    threshold that keeps all of the top K and few others; a second pass
//    compacts the slots at or above it into items.
// 2. MSB-first radix select on the composite, one byte per pass, starting
//    at the highest nonzero byte of p: inside one 1024-thread block for
//    short lists; otherwise across the grid, where each pass histograms the
//    surviving tie set, the last block to finish picks the byte, and the
//    next pass keeps only the survivors with that byte (passes whose work is
//    already decided exit at once, so the host never waits between passes).
// 3. Collection: every item whose composite is at least the threshold.
// 4. Bitonic sort of the K items (shared-memory stages inside 2048-item
//    chunks, global stages across chunks).
#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <cmath>
#include <vector>

#include "mad_device.cuh"
#include "mad_internal.cuh"

namespace mad {
namespace {

struct SelState {
  unsigned int lhist[1024];   // log-bucket histogram of x (hash path)
  unsigned long long theta;   // collect threshold from the histogram
  unsigned long long maxp;
  unsigned long long positive;
  unsigned int ticket3;
  unsigned int pad3;
  unsigned long long n_cur;   // survivors in the current list
  unsigned long long k_rem;   // survivors still to be taken
  unsigned long long tp, tk;  // threshold composite (tk applies to ~key)
  unsigned long long n_next;
  unsigned int hist[256];
  unsigned int ticket;
  unsigned int ticket2;
  int cur;                    // 0: the compacted list, 1/2: ping-pong lists
  int done;
  int picked;
  int pad;
};

__device__ __forceinline__ uint32_t digit_of(const Item& it, int q, int dp) {
  if (q < dp) return (uint32_t)(it.p >> (8 * (dp - 1 - q))) & 0xFFu;
  return (uint32_t)((~it.key) >> (8 * (7 - (q - dp)))) & 0xFFu;
}

// Warp-aggregated append of `it` when `want` (one counter atomic per warp
// that holds an item: the cheaper form when few warps do).
__device__ __forceinline__ void append_warp(Item* out, unsigned long long* counter, bool want,
                                            const Item& it, uint64_t cap) {
  const unsigned mask = __ballot_sync(0xFFFFFFFFu, want);
  if (!mask) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (want) {
    const unsigned long long pos = base + __popc(mask & ((1u << lane) - 1u));
    if (pos < cap) out[pos] = it;
  }
}

// Block-wide append of up to N items per thread: every thread of the block
// calls it the same number of times.  One atomic on the counter per block
// and call (a single counter shared by every warp of the grid serialises
// when most warps hold an item, as 0/1 counts near the threshold do).
template <int N>
__device__ __forceinline__ void append_block(Item* out, unsigned long long* counter,
                                             const bool (&want)[N], const Item (&it)[N],
                                             uint64_t cap) {
  __shared__ unsigned int s_cnt[32];
  __shared__ unsigned long long s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned mask[N];
  unsigned total = 0;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    mask[q] = __ballot_sync(0xFFFFFFFFu, want[q]);
    total += __popc(mask[q]);
  }
  if (lane == 0) s_cnt[warp] = total;
  __syncthreads();
  if (warp == 0) {
    const int nw = (int)(blockDim.x >> 5);
    unsigned v = lane < nw ? s_cnt[lane] : 0u;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned u = __shfl_up_sync(0xFFFFFFFFu, v, off);
      if (lane >= off) v += u;
    }
    if (lane < nw) s_cnt[lane] = v;   // inclusive, per warp
    if (lane == 31) s_base = v ? atomicAdd(counter, (unsigned long long)v) : 0ull;
  }
  __syncthreads();
  unsigned long long pos = s_base + (warp ? s_cnt[warp - 1] : 0u);
  const unsigned below = (1u << lane) - 1u;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    if (want[q]) {
      const unsigned long long p = pos + __popc(mask[q] & below);
      if (p < cap) out[p] = it[q];
    }
    pos += __popc(mask[q]);
  }
  __syncthreads();   // s_cnt and s_base are reused by the next call
}

__device__ __forceinline__ void append_block1(Item* out, unsigned long long* counter, bool want,
                                              const Item& it, uint64_t cap) {
  const bool w[1] = {want};
  const Item v[1] = {it};
  append_block<1>(out, counter, w, v, cap);
}

__global__ void __launch_bounds__(256)
k_radix_hist(const Item* __restrict__ l0, const Item* __restrict__ l1,
             const Item* __restrict__ l2, SelState* st, int q, int dp, int last_q) {
  if (st->done) return;
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const Item* list = st->cur == 0 ? l0 : (st->cur == 1 ? l1 : l2);
  const unsigned long long n = st->n_cur;
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (unsigned long long)gridDim.x * blockDim.x)
    atomicAdd(&h[digit_of(list[x], q, dp)], 1u);
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&st->hist[threadIdx.x], h[threadIdx.x]);
  __threadfence();
  __shared__ unsigned int is_last;
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    volatile unsigned int* gh = st->hist;
    unsigned long long above = 0;
    int b = 255;
    for (; b > 0; --b) {
      const unsigned long long c = gh[b];
      if (above + c >= st->k_rem) break;
      above += c;
    }
    const unsigned long long ties = gh[b];
    st->k_rem -= above;
    st->picked = b;
    if (q < dp)
      st->tp |= (unsigned long long)b << (8 * (dp - 1 - q));
    else
      st->tk |= (unsigned long long)b << (8 * (7 - (q - dp)));
    // Every survivor with this byte is taken, or the threshold is complete.
    if (ties == st->k_rem || q == last_q) st->done = 1;
    st->ticket = 0;
    st->n_next = 0;
  }
  __syncthreads();
  st->hist[threadIdx.x] = 0;
}

__global__ void __launch_bounds__(256)
k_radix_filter(const Item* __restrict__ l0, Item* __restrict__ l1, Item* __restrict__ l2,
               SelState* st, int q, int dp, uint64_t cap) {
  if (st->done) return;
  const int cur = st->cur;
  const Item* list = cur == 0 ? l0 : (cur == 1 ? l1 : l2);
  Item* out = cur == 1 ? l2 : l1;
  const unsigned long long n = st->n_cur;
  const uint32_t picked = (uint32_t)st->picked;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long rounds = (n + stride - 1) / stride;
  for (unsigned long long r = 0; r < rounds; ++r) {
    const unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x + r * stride;
    bool want = false;
    Item it;
    if (x < n) {
      it = list[x];
      want = digit_of(it, q, dp) == picked;
    }
    append_block1(out, &st->n_next, want, it, cap);
  }
  __threadfence();
  __shared__ unsigned int is_last;
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->ticket2, 1u) == gridDim.x - 1);
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    st->cur = cur == 1 ? 2 : 1;
    st->n_cur = *((volatile unsigned long long*)&st->n_next);
    st->ticket2 = 0;
  }
}

__global__ void __launch_bounds__(256)
k_collect(const Item* __restrict__ l0, unsigned long long n, const SelState* st,
          Item* __restrict__ out, unsigned long long* counter, uint64_t cap) {
  const unsigned long long tp = st->tp, tk = st->tk;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long rounds = (n + stride - 1) / stride;
  for (unsigned long long r = 0; r < rounds; ++r) {
    const unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x + r * stride;
    bool want = false;
    Item it;
    if (x < n) {
      it = l0[x];
      want = it.p > tp || (it.p == tp && (~it.key) >= tk);
    }
    append_block1(out, counter, want, it, cap);
  }
}

// ---- hash path: one-pass log-bucket histogram, then a threshold compaction --
// Bucket of v >= 1: 16 * floor(log2 v) + the 4 bits below the leading bit
// (1024 buckets, monotone in v).  The collect threshold is the lower bound
// of the bucket in which the count from the top reaches K, so at least K
// items (all of the top K) pass and few more do.

// With lg > 0 only every 2^lg-th group of 4 slots (one 32-byte sector of
// values) is read, and the bucket picked is where the sampled count from the
// top reaches K (the caller scales K to the sample).  With a gate, the
// kernel runs only when *gate is nonzero.
__global__ void __launch_bounds__(256)
k_log_hist(const long long* __restrict__ vals, uint64_t cap_max, unsigned long long K,
           SelState* st, const unsigned long long* cap_dev, int lg = 0,
           const unsigned int* gate = nullptr) {
  if (gate && *gate == 0u) return;
  const uint64_t cap = dev_len(cap_max, cap_dev);
  const uint64_t groups = (cap + 3) >> 2;
  const uint64_t span = ((groups + (1ull << lg) - 1) >> lg) << 2;   // sampled slots
  __shared__ unsigned int h[1024];
  for (int b = threadIdx.x; b < 1024; b += blockDim.x) h[b] = 0;
  __syncthreads();
  unsigned long long mx = 0;
  // Four independent loads per thread per round keep enough bytes in flight.
  constexpr int U = 4;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t rounds = (span + U * stride - 1) / (U * stride);
  for (uint64_t r = 0; r < rounds; ++r) {
    long long v[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const uint64_t x = (r * U + q) * stride + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
      const uint64_t slot = (((x >> 2) << lg) << 2) | (x & 3);
      v[q] = slot < cap ? __ldg(vals + slot) : 0;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      // (a shared-memory atomic per value measured faster than combining
      // equal buckets of a warp first)
      if (v[q] > 0) {
        atomicAdd(&h[log_bucket((unsigned long long)v[q])], 1u);
        if ((unsigned long long)v[q] > mx) mx = (unsigned long long)v[q];
      }
    }
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, mx, off);
    mx = o > mx ? o : mx;
  }
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(&st->maxp, mx);
  __syncthreads();
  for (int b = threadIdx.x; b < 1024; b += blockDim.x)
    if (h[b]) atomicAdd(&st->lhist[b], h[b]);
  __threadfence();
  __shared__ unsigned int is_last;
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->ticket3, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  unsigned long long total = 0;
  const int b = block_pick_from_top<1024>(st->lhist, K, &total);
  if (threadIdx.x == 0) {
    st->theta = b >= 0 ? bucket_floor((uint32_t)b) : 1ull;  // fewer than K positive: take all
    st->positive = total;
  }
}

// kBlock: one counter atomic per block and round (0/1 inputs: their small
// counts tie at the threshold, so most warps of 32 slots hold an item and
// per-warp atomics on the one counter serialise); otherwise one atomic per
// warp that holds an item (dense inputs: a thin band of slots passes).
template <bool kBlock>
__global__ void __launch_bounds__(256)
k_compact_ge(const unsigned long long* __restrict__ keys, const long long* __restrict__ vals,
             uint64_t cap_max, const SelState* st, Item* __restrict__ out, uint64_t out_cap,
             unsigned long long* counter, const unsigned long long* cap_dev,
             const unsigned int* gate = nullptr) {
  if (gate && *gate == 0u) return;
  const uint64_t cap = dev_len(cap_max, cap_dev);
  const unsigned long long theta = st->theta;
  constexpr int U = 4;   // independent loads in flight per thread
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t rounds = (cap + U * stride - 1) / (U * stride);
  const uint64_t start = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (uint64_t r = 0; r < rounds; ++r) {
    long long v[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const uint64_t slot = start + (r * U + q) * stride;
      v[q] = slot < cap ? __ldcs(vals + slot) : 0;
    }
    if (kBlock) {   // the round's U items of every thread in one block-wide append
      bool want[U];
      Item it[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const uint64_t slot = start + (r * U + q) * stride;
        want[q] = v[q] > 0 && (unsigned long long)v[q] >= theta;
        if (want[q]) {
          it[q].p = (unsigned long long)v[q];
          it[q].key = keys[slot];
          it[q].aux = slot;
        }
      }
      append_block<U>(out, counter, want, it, out_cap);
    } else {
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const uint64_t slot = start + (r * U + q) * stride;
        const bool want = v[q] > 0 && (unsigned long long)v[q] >= theta;
        Item it;
        if (want) {
          it.p = (unsigned long long)v[q];
          it.key = keys[slot];
          it.aux = slot;
        }
        append_warp(out, counter, want, it, out_cap);
      }
    }
  }
}

// k_compact_ge in the append mode of the context's inputs.
template <typename... Args>
void launch_compact_ge(const mad_ctx* ctx, unsigned blocks, cudaStream_t st, Args... args) {
  if (ctx->integer) k_compact_ge<true><<<blocks, 256, 0, st>>>(args...);
  else k_compact_ge<false><<<blocks, 256, 0, st>>>(args...);
}

// After a compaction at a threshold estimated from a sample: when it kept
// fewer than K items although the threshold excluded some (theta > 1),
// *gate is set and the state is reset for the exact histogram and
// compaction, which run gated on it.
__global__ void __launch_bounds__(256)
k_select_check(SelState* st, unsigned long long* counter, unsigned long long K,
               unsigned int* gate) {
  __shared__ int redo;
  if (threadIdx.x == 0) {
    redo = (*counter < K && st->theta > 1ull) ? 1 : 0;
    *gate = (unsigned int)redo;
  }
  __syncthreads();
  if (!redo) return;
  for (int b = threadIdx.x; b < 1024; b += blockDim.x) st->lhist[b] = 0;
  if (threadIdx.x == 0) {
    *counter = 0;
    st->ticket3 = 0;
    st->maxp = 0;
    st->positive = 0;
  }
}

// ---- tile sort + merge rank (lists up to 2^17 items) ------------------------
// Total order: p desc, key asc, then input position asc (so repeated keys
// still get distinct ranks).  Step 1 sorts tiles of 2048 items in shared
// memory (bitonic network); step 2 gives every item whose rank inside its
// tile is below K its global rank, its tile rank plus, for every other tile,
// the number of that tile's items ordered before it (a binary search), and
// writes the items ranked below K to their place.
constexpr unsigned kTile = 2048;
constexpr unsigned kTileSortMax = 1u << 17;
// One-block selection (k_block_select, below): lists up to kBlockSel items,
// sorted output up to kBlockSort items.
constexpr int kBlockSel = 16384;
constexpr int kBlockSort = 2048;

__device__ __forceinline__ bool item_before(unsigned long long ap, unsigned long long ak, uint32_t ai,
                                            unsigned long long bp, unsigned long long bk, uint32_t bi) {
  return ap > bp || (ap == bp && (ak < bk || (ak == bk && ai < bi)));
}

__global__ void __launch_bounds__(1024)
k_tile_sort(const Item* __restrict__ in, unsigned n_max, unsigned K, Item* __restrict__ out,
            uint32_t* __restrict__ pos_out, const unsigned long long* n_dev,
            unsigned int* over_err, const unsigned int* gate = nullptr) {
  __shared__ unsigned long long sp[kTile], sk[kTile];
  __shared__ uint32_t si[kTile];
  if (gate && *gate == 0u) return;   // the list was selected by k_block_select
  // Under a device count: a list longer than the workspace is reported.
  if (over_err && blockIdx.x == 0 && threadIdx.x == 0 && *n_dev > n_max)
    atomicOr(over_err, DERR_SELECT);
  const unsigned n = (unsigned)dev_len(n_max, n_dev);
  const unsigned base = blockIdx.x * kTile;
  if (base >= n) return;
  const unsigned len = min(kTile, n - base);
  for (unsigned r = threadIdx.x; r < kTile; r += blockDim.x) {
    if (r < len) {
      sp[r] = in[base + r].p;
      sk[r] = in[base + r].key;
      si[r] = base + r;
    } else {
      sp[r] = 0;
      sk[r] = ~0ull;
      si[r] = 0xFFFFFFFFu;
    }
  }
  __syncthreads();
  for (unsigned k = 2; k <= kTile; k <<= 1) {
    for (unsigned j = k >> 1; j > 0; j >>= 1) {
      const unsigned t = threadIdx.x;   // kTile / 2 compare-exchanges
      const unsigned a = ((t & ~(j - 1)) << 1) | (t & (j - 1)), b = a + j;   // j a power of two
      const bool up = (a & k) == 0;
      const bool b_first = item_before(sp[b], sk[b], si[b], sp[a], sk[a], si[a]);
      if (b_first == up) {
        const unsigned long long tp = sp[a], tk = sk[a];
        const uint32_t ti = si[a];
        sp[a] = sp[b]; sk[a] = sk[b]; si[a] = si[b];
        sp[b] = tp; sk[b] = tk; si[b] = ti;
      }
      __syncthreads();
    }
  }
  for (unsigned r = threadIdx.x; r < len; r += blockDim.x) {
    if (pos_out) {
      out[base + r] = in[si[r]];
      pos_out[base + r] = si[r];
    } else if (r < K) {
      out[r] = in[si[r]];
    }
  }
}

__global__ void __launch_bounds__(256)
k_merge_rank(const Item* __restrict__ tiles, const uint32_t* __restrict__ pos, unsigned n_max,
             unsigned K, Item* __restrict__ out, const unsigned long long* n_dev,
             const unsigned int* gate = nullptr) {
  if (gate && *gate == 0u) return;
  const unsigned n = (unsigned)dev_len(n_max, n_dev);
  const unsigned x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  const unsigned my_tile = x / kTile, r = x % kTile;
  if (r >= K) return;
  const Item me = tiles[x];
  const uint32_t mi = pos[x];
  const unsigned ntiles = (n + kTile - 1) / kTile;
  unsigned rank = r;
  for (unsigned b = 0; b < ntiles && rank < K; ++b) {
    if (b == my_tile) continue;
    const unsigned base = b * kTile, len = min(kTile, n - base);
    unsigned lo = 0, cnt = len;   // first entry of tile b not ordered before me
    while (cnt > 0) {
      const unsigned half = cnt >> 1, q = base + lo + half;
      if (item_before(tiles[q].p, tiles[q].key, pos[q], me.p, me.key, mi)) {
        lo += half + 1;
        cnt -= half + 1;
      } else {
        cnt = half;
      }
    }
    rank += lo;
  }
  if (rank < K) out[rank] = me;
}

// Pairwise merge of sorted runs of length L (kTile times a power of two):
// item x of run R goes to (R & ~1) L + its rank inside R + the number of
// items of the partner run R ^ 1 ordered before it (a binary search; the
// order is total, so the places are distinct).
__global__ void __launch_bounds__(256)
k_merge_pairs(const Item* __restrict__ in, const uint32_t* __restrict__ pin, unsigned n,
              unsigned L, Item* __restrict__ out, uint32_t* __restrict__ pout) {
  const unsigned x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  const unsigned R = x / L, r = x - R * L;
  const unsigned pb = (R ^ 1u) * L;
  const Item me = in[x];
  const uint32_t mi = pin[x];
  unsigned lo = 0;
  if (pb < n) {
    unsigned cnt = min(L, n - pb);
    while (cnt > 0) {
      const unsigned half = cnt >> 1, q = pb + lo + half;
      if (item_before(in[q].p, in[q].key, pin[q], me.p, me.key, mi)) {
        lo += half + 1;
        cnt -= half + 1;
      } else {
        cnt = half;
      }
    }
  }
  const unsigned dst = (R & ~1u) * L + r + lo;
  out[dst] = me;
  pout[dst] = mi;
}

// Every item of in[0..n) sorted into ws.out (kTile < n <= kTileSortMax):
// tiles sorted in shared memory, then log2(tiles) rounds of pairwise
// merges.  Items alternate between ws.l1 and ws.out, their input positions
// between the two halves of ws.l2; `in` may be ws.out.
void sort_merge(mad_ctx* ctx, const SelectWs& ws, const Item* in, uint64_t n, cudaStream_t st) {
  const unsigned tiles = (unsigned)((n + kTile - 1) / kTile);
  int rounds = 0;
  while ((1u << rounds) < tiles) ++rounds;
  uint32_t* pa = (uint32_t*)ws.l2;
  uint32_t* pb = pa + n;
  // The buffer the tile sort writes, so that the last round lands in ws.out
  // (ws.l1 when `in` is ws.out itself, then one copy at the end).
  Item* cur = (rounds % 2 == 0 && in != ws.out) ? ws.out : ws.l1;
  Item* other = cur == ws.out ? ws.l1 : ws.out;
  k_tile_sort<<<tiles, kTile / 2, 0, st>>>(in, (unsigned)n, (unsigned)n, cur, pa, nullptr,
                                            nullptr);
  count_launch(ctx);
  const unsigned blocks = (unsigned)((n + 255) / 256);
  for (int r = 0; r < rounds; ++r) {
    k_merge_pairs<<<blocks, 256, 0, st>>>(cur, pa, (unsigned)n, kTile << r, other, pb);
    count_launch(ctx);
    Item* t = cur;
    cur = other;
    other = t;
    uint32_t* u = pa;
    pa = pb;
    pb = u;
  }
  if (cur != ws.out) cudaMemcpyAsync(ws.out, cur, n * sizeof(Item), cudaMemcpyDeviceToDevice, st);
}

// Sorted top K of `in[0..n)` by tiles (n <= kTileSortMax).  Uses l1 and l2
// of the workspace as scratch; `in` may be ws.out.
void tile_select(mad_ctx* ctx, const SelectWs& ws, const Item* in, uint64_t n, uint64_t K,
                 cudaStream_t st) {
  const unsigned tiles = (unsigned)((n + kTile - 1) / kTile);
  if (tiles == 1 && in != ws.out) {
    k_tile_sort<<<1, kTile / 2, 0, st>>>(in, (unsigned)n, (unsigned)K, ws.out, nullptr, nullptr,
                                         nullptr);
    count_launch(ctx);
    return;
  }
  uint32_t* pos = (uint32_t*)ws.l2;
  k_tile_sort<<<tiles, kTile / 2, 0, st>>>(in, (unsigned)n, (unsigned)K, ws.l1, pos, nullptr,
                                            nullptr);
  k_merge_rank<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ws.l1, pos, (unsigned)n, (unsigned)K,
                                                            ws.out, nullptr);
  count_launch(ctx, 2);
}

// ---- bitonic sort: "before" = (p desc, key asc) --------------------------
__device__ __forceinline__ bool before(const Item& a, const Item& b) {
  return a.p > b.p || (a.p == b.p && a.key < b.key);
}

__device__ __forceinline__ void cmp_swap(Item& a, Item& b, bool up) {
  // up: a must come before b.
  const bool sw = up ? before(b, a) : before(a, b);
  if (sw) {
    const Item t = a;
    a = b;
    b = t;
  }
}

constexpr int SORT_CHUNK = 2048;

__global__ void __launch_bounds__(256)
k_bitonic_local(Item* data, unsigned long long n2, int chunk, int full_sort,
                unsigned long long kk) {
  extern __shared__ Item sm[];
  const unsigned long long base = (unsigned long long)blockIdx.x * chunk;
  for (int t = threadIdx.x; t < chunk; t += blockDim.x) sm[t] = data[base + t];
  __syncthreads();
  if (full_sort) {
    for (int k = 2; k <= chunk; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < chunk; t += blockDim.x) {
          const int l = t ^ j;
          if (l > t) cmp_swap(sm[t], sm[l], ((base + t) & (unsigned long long)k) == 0);
        }
        __syncthreads();
      }
    }
  } else {
    for (int j = chunk >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < chunk; t += blockDim.x) {
        const int l = t ^ j;
        if (l > t) cmp_swap(sm[t], sm[l], ((base + t) & kk) == 0);
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < chunk; t += blockDim.x) data[base + t] = sm[t];
}

__global__ void __launch_bounds__(256)
k_bitonic_global(Item* data, unsigned long long n2, unsigned long long k, unsigned long long j) {
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n2) return;
  const unsigned long long l = t ^ j;
  if (l > t) cmp_swap(data[t], data[l], (t & k) == 0);
}

__global__ void k_pad(Item* data, unsigned long long from, unsigned long long to) {
  const unsigned long long t = from + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < to) {
    Item s;
    s.p = 0;
    s.key = ~0ull;
    s.aux = ~0ull;
    data[t] = s;
  }
}

__global__ void k_to_pairs(const Item* __restrict__ items, unsigned long long n_max,
                           const mad_pair* __restrict__ cand, const double* __restrict__ cvals,
                           mad_pair* __restrict__ out, const unsigned long long* n_dev,
                           uint32_t* n_out) {
  const unsigned long long n = dev_len(n_max, n_dev);
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n_out && t == 0) *n_out = (uint32_t)n;
  if (t >= n) return;
  const Item it = items[t];
  mad_pair pr;
  pr.i = (uint32_t)(it.key >> 32);
  pr.j = (uint32_t)it.key;
  if (cand) {
    pr.x = cand[it.aux].x;
    pr.c = cvals[it.aux];
  } else {
    pr.x = (int64_t)it.p;
    pr.c = 0.0;
  }
  out[t] = pr;
}

unsigned grid_for(unsigned long long n, unsigned cap_blocks) {
  const unsigned long long b = (n + 255) / 256;
  return (unsigned)(b == 0 ? 1 : (b < cap_blocks ? b : cap_blocks));
}

void bitonic_sort(mad_ctx* ctx, Item* data, unsigned long long n, cudaStream_t st,
                  unsigned long long* n2_out) {
  unsigned long long n2 = 2;
  while (n2 < n) n2 <<= 1;
  *n2_out = n2;
  if (n2 > n) {
    k_pad<<<grid_for(n2 - n, 1u << 20), 256, 0, st>>>(data, n, n2);
    count_launch(ctx);
  }
  const int chunk = (int)(n2 < (unsigned long long)SORT_CHUNK ? n2 : SORT_CHUNK);
  const unsigned blocks = (unsigned)(n2 / chunk);
  const size_t smem = (size_t)chunk * sizeof(Item);
  k_bitonic_local<<<blocks, 256, smem, st>>>(data, n2, chunk, 1, 0);
  count_launch(ctx);
  for (unsigned long long k = 2ull * chunk; k <= n2; k <<= 1) {
    for (unsigned long long j = k >> 1; j >= (unsigned long long)chunk; j >>= 1) {
      k_bitonic_global<<<grid_for(n2, 1u << 30), 256, 0, st>>>(data, n2, k, j);
      count_launch(ctx);
    }
    k_bitonic_local<<<blocks, 256, smem, st>>>(data, n2, chunk, 0, k);
    count_launch(ctx);
  }
}

}  // namespace

int significant_bytes(unsigned long long maxp) {
  int b = 1;
  while (b < 8 && (maxp >> (8 * b)) != 0) ++b;
  return b;
}

size_t select_ws_bytes(uint64_t n, uint64_t K) {
  uint64_t n2 = 2;
  while (n2 < (K < n ? K : n)) n2 <<= 1;
  const uint64_t lists = 3 * (n ? n : 1);
  return (lists + n2) * sizeof(Item) + sizeof(SelState) + 4 * sizeof(unsigned long long) + 256;
}

SelectWs select_ws_carve(void* base, uint64_t n, uint64_t K) {
  uint64_t n2 = 2;
  while (n2 < (K < n ? K : n)) n2 <<= 1;
  SelectWs ws;
  const uint64_t nn = n ? n : 1;
  ws.l0 = (Item*)base;
  ws.l1 = ws.l0 + nn;
  ws.l2 = ws.l1 + nn;
  ws.out = ws.l2 + nn;
  ws.state = (void*)(ws.out + n2);
  ws.counter = (unsigned long long*)((char*)ws.state + ((sizeof(SelState) + 255) / 256) * 256);
  ws.cap_n = nn;
  ws.cap_out = n2;
  return ws;
}

void prefilter_select(mad_ctx* ctx, const SelectWs& ws, uint64_t n, uint64_t K, cudaStream_t st);

mad_status select_list(mad_ctx* ctx, const SelectWs& ws, uint64_t n, uint64_t K, int dp,
                       uint64_t* n_sel, cudaStream_t st) {
  const uint64_t take = K < n ? K : n;
  *n_sel = take;
  if (take == 0) return MAD_OK;
  unsigned long long n2 = 0;
  // Lists up to 2^17 items go straight to the tile sort.  Longer ones first
  // pick the K largest, unordered, into ws.out (an MSB radix select), which
  // the tile sort then orders when K is short, else a bitonic network.
  if (n <= kTileSortMax) {
    if (take <= (uint64_t)kBlockSort && take < n && n > (uint64_t)kTile)
      prefilter_select(ctx, ws, n, take, st);
    else if (take == n && n > (uint64_t)kTile)
      sort_merge(ctx, ws, ws.l0, n, st);
    else
      tile_select(ctx, ws, ws.l0, n, take, st);
    return cuda_status(cudaGetLastError());
  }
  if (take == n) {
    cudaMemcpyAsync(ws.out, ws.l0, n * sizeof(Item), cudaMemcpyDeviceToDevice, st);
  } else {
    SelState* dst = (SelState*)ws.state;
    cudaMemsetAsync(dst, 0, sizeof(SelState), st);
    const unsigned long long init[2] = {n, K};
    cudaMemcpyAsync(&dst->n_cur, init, sizeof(init), cudaMemcpyHostToDevice, st);
    const int digits = dp + 8;
    const unsigned blocks = grid_for(n, 152 * 4);
    for (int q = 0; q < digits; ++q) {
      k_radix_hist<<<blocks, 256, 0, st>>>(ws.l0, ws.l1, ws.l2, dst, q, dp, digits - 1);
      k_radix_filter<<<blocks, 256, 0, st>>>(ws.l0, ws.l1, ws.l2, dst, q, dp, ws.cap_n);
      count_launch(ctx, 2);
    }
    cudaMemsetAsync(ws.counter, 0, sizeof(unsigned long long), st);
    k_collect<<<grid_for(n, 152 * 8), 256, 0, st>>>(ws.l0, n, dst, ws.out, ws.counter, ws.cap_out);
    count_launch(ctx);
  }
  if (take <= kTileSortMax) {
    if (take > (uint64_t)kTile) sort_merge(ctx, ws, ws.out, take, st);
    else tile_select(ctx, ws, ws.out, take, take, st);
    return cuda_status(cudaGetLastError());
  }
  bitonic_sort(ctx, ws.out, take, st, &n2);
  return cuda_status(cudaGetLastError());
}

mad_status select_from_hash(mad_ctx* ctx, const SelectWs& ws, uint64_t K, uint64_t* n_sel,
                            uint64_t* n_pos, cudaStream_t st) {
  SelState* dst = (SelState*)ws.state;
  cudaMemsetAsync(dst, 0, sizeof(SelState), st);
  cudaMemsetAsync(ws.counter, 0, sizeof(unsigned long long), st);
  const uint64_t bound = hash_slot_bound(ctx);
  const unsigned blocks = grid_for(bound, 152 * 8);
  const unsigned long long* extent = hash_extent(ctx);
  k_log_hist<<<blocks, 256, 0, st>>>(ctx->hvals, bound, K, dst, extent);
  launch_compact_ge(ctx, blocks, st, ctx->hkeys, ctx->hvals, bound, dst, ws.l0, ws.cap_n,
                    ws.counter, extent);
  count_launch(ctx, 2);
  unsigned long long host[2] = {0, 0};
  cudaMemcpyAsync(&host[0], ws.counter, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&host[1], &dst->maxp, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
  unsigned long long positive = 0;
  cudaMemcpyAsync(&positive, &dst->positive, sizeof(positive), cudaMemcpyDeviceToHost, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  if (host[0] > ws.cap_n) return MAD_ERR_STATE;
  *n_pos = positive;
  return select_list(ctx, ws, host[0], K, significant_bytes(host[1]), n_sel, st);
}

mad_status items_to_pairs(mad_ctx* ctx, const Item* items, uint64_t n, const mad_pair* cand,
                          const double* cvals, mad_pair* out, cudaStream_t st) {
  if (n == 0) return MAD_OK;
  k_to_pairs<<<grid_for(n, 1u << 30), 256, 0, st>>>(items, n, cand, cvals, out, nullptr, nullptr);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

void tile_select_dev(mad_ctx* ctx, const Item* in, uint64_t cap, uint64_t K,
                     const unsigned long long* n_dev, unsigned int* over_err, Item* sorted,
                     uint32_t* pos, Item* out, cudaStream_t st, const unsigned int* gate) {
  const unsigned tiles = (unsigned)((cap + kTile - 1) / kTile);
  k_tile_sort<<<tiles, kTile / 2, 0, st>>>(in, (unsigned)cap, (unsigned)K, sorted, pos, n_dev,
                                            over_err, gate);
  k_merge_rank<<<(unsigned)((cap + 255) / 256), 256, 0, st>>>(sorted, pos, (unsigned)cap,
                                                              (unsigned)K, out, n_dev, gate);
  count_launch(ctx, 2);
}

// ---- one-block exact selection ---------------------------------------------
// The K largest of the first n = min(cap, *n_dev) items by (p desc, key
// asc), for n <= kBlockSel, in one 1024-thread block: the p of every item
// sit in shared memory and an MSB radix select (8-bit digits, from the
// highest digit in which two items differ) finds the K-th largest p and how
// many items equal to it are taken; among those
// ties the smallest keys are found the same way.  The K items go to out in
// no particular order, or sorted when `sorted` (K <= kBlockSort).  A longer
// list sets *gate to 1 and writes nothing (the tile kernels, gated on that
// word, select instead); otherwise *gate becomes 0.

// The digit of the K-th largest value among those counted in hist (256
// bins, digit order): returns it and leaves in *rank the rank of that value
// inside its digit (from the top).  One warp.
__device__ __forceinline__ void pick_digit(const unsigned int* hist, unsigned long long* rank,
                                           int* digit) {
  const int lane = threadIdx.x & 31;
  // lane L holds bins 255 - 8L ... 248 - 8L (from the top)
  unsigned int c[8];
  unsigned int mine = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    c[u] = hist[255 - 8 * lane - u];
    mine += c[u];
  }
  unsigned int inc = mine;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned int o = __shfl_up_sync(0xFFFFFFFFu, inc, off);
    if (lane >= off) inc += o;
  }
  const unsigned long long need = *rank;
  const unsigned long long before = inc - mine;
  const bool here = before < need && (unsigned long long)inc >= need;
  const unsigned who = __ballot_sync(0xFFFFFFFFu, here);
  if (here) {
    unsigned long long cum = before;
    for (int u = 0; u < 8; ++u) {
      if (cum + c[u] >= need) {
        *digit = 255 - 8 * lane - u;
        *rank = need - cum;
        break;
      }
      cum += c[u];
    }
  }
  (void)who;
}

__global__ void __launch_bounds__(1024)
k_block_select(const Item* __restrict__ in, unsigned long long cap, const unsigned long long* n_dev,
               unsigned int K_max, Item* __restrict__ out, int sorted, unsigned int* gate) {
  extern __shared__ unsigned long long bs_p[];   // kBlockSel values, then the sort buffers
  __shared__ unsigned int hist[256];
  __shared__ unsigned long long s_prefix, s_rank, s_kprefix, s_krank, s_diff;
  __shared__ int s_digit;
  __shared__ unsigned int s_out, s_tie;
  const unsigned long long n = dev_len(cap, n_dev);
  if (n > (unsigned long long)kBlockSel) {
    if (threadIdx.x == 0) *gate = 1u;
    return;
  }
  const unsigned long long K = (unsigned long long)K_max < n ? (unsigned long long)K_max : n;
  // The bits in which the items differ from the first one: the digits
  // above the highest of them are the same in every item and need no pass.
  const unsigned long long v0 = n > 0 ? in[0].p : 0ull;
  unsigned long long diff = 0;
  for (unsigned long long x = threadIdx.x; x < n; x += blockDim.x) {
    const unsigned long long v = in[x].p;
    bs_p[x] = v;
    diff |= v ^ v0;
  }
  if (threadIdx.x == 0) {
    s_diff = 0;
    s_out = 0;
    s_tie = 0;
  }
  __syncthreads();
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) diff |= __shfl_xor_sync(0xFFFFFFFFu, diff, off);
  if ((threadIdx.x & 31) == 0 && diff) atomicOr(&s_diff, diff);
  __syncthreads();
  // First digit that can differ (-1: all items equal).
  const int d_top = s_diff ? (63 - __clzll((long long)s_diff)) / 8 : -1;
  unsigned long long mask = d_top >= 7 ? 0ull : ~0ull << (8 * (d_top + 1));
  if (threadIdx.x == 0) {
    s_prefix = v0 & mask;
    s_rank = K;
  }
  __syncthreads();
  // MSB radix select of the K-th largest p.
  for (int d = d_top; d >= 0 && K > 0; --d) {
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const unsigned long long prefix = s_prefix;
    for (unsigned long long x = threadIdx.x; x < n; x += blockDim.x) {
      const unsigned long long v = bs_p[x];
      if ((v & mask) == prefix) atomicAdd(&hist[(v >> (8 * d)) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      unsigned long long r = s_rank;
      int dg = -1;
      pick_digit(hist, &r, &dg);
      if (dg >= 0) {   // exactly one lane found the digit
        s_digit = dg;
        s_rank = r;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_prefix = prefix | ((unsigned long long)s_digit << (8 * d));
    mask |= 255ull << (8 * d);
    __syncthreads();
  }
  const unsigned long long pk = s_prefix;          // the K-th largest p
  const unsigned long long take_ties = s_rank;     // items equal to pk that are taken
  // Ties: the take_ties smallest keys among the items with p == pk.
  unsigned long long tie_count = 0;
  for (unsigned long long x = threadIdx.x; x < n; x += blockDim.x) tie_count += bs_p[x] == pk;
  atomicAdd(&s_tie, (unsigned int)tie_count);
  if (threadIdx.x == 0) {
    s_kprefix = ~0ull;   // every tied key qualifies unless a key threshold is set
    s_krank = take_ties;
  }
  __syncthreads();
  const bool key_select = K > 0 && take_ties < s_tie;
  if (key_select) {
    // MSB radix select of the take_ties-th smallest key among the ties:
    // ranks from the top of ~key.
    if (threadIdx.x == 0) s_kprefix = 0;
    __syncthreads();
    unsigned long long kmask = 0;
    for (int d = 7; d >= 0; --d) {
      for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
      __syncthreads();
      const unsigned long long kp = s_kprefix;
      for (unsigned long long x = threadIdx.x; x < n; x += blockDim.x) {
        if (bs_p[x] != pk) continue;
        const unsigned long long nk = ~in[x].key;
        if ((nk & kmask) == kp) atomicAdd(&hist[(nk >> (8 * d)) & 255u], 1u);
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        unsigned long long r = s_krank;
        int dg = -1;
        pick_digit(hist, &r, &dg);
        if (dg >= 0) {
          s_digit = dg;
          s_krank = r;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_kprefix = kp | ((unsigned long long)s_digit << (8 * d));
      kmask |= 255ull << (8 * d);
      __syncthreads();
    }
  }
  const unsigned long long nk_min = s_kprefix;   // taken ties have ~key >= this
  // The selected items (their p values are still in shared memory).
  const bool to_smem = sorted && K <= (unsigned long long)kBlockSort;
  __syncthreads();
  unsigned long long* sp = bs_p + kBlockSel;   // sort buffers after the values
  for (unsigned long long x = threadIdx.x; x < n; x += blockDim.x) {
    const unsigned long long v = bs_p[x];
    bool take = K > 0 && v > pk;
    if (!take && K > 0 && v == pk) take = !key_select || ~in[x].key >= nk_min;
    if (take) {
      const unsigned int pos = atomicAdd(&s_out, 1u);
      if (pos >= K) continue;   // (never: exactly K items qualify)
      if (to_smem) {
        sp[pos] = v;
        sp[kBlockSort + pos] = in[x].key;
        sp[2 * kBlockSort + pos] = in[x].aux;
      } else {
        out[pos] = in[x];
      }
    }
  }
  __syncthreads();
  if (to_smem) {
    const int m = (int)K;
    int m2 = 1;
    while (m2 < m) m2 <<= 1;
    for (int x = m + threadIdx.x; x < m2; x += blockDim.x) {
      sp[x] = 0;
      sp[kBlockSort + x] = ~0ull;
      sp[2 * kBlockSort + x] = 0;
    }
    __syncthreads();
    unsigned long long* kk = sp + kBlockSort;
    unsigned long long* aa = sp + 2 * kBlockSort;
    for (int k = 2; k <= m2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < m2 / 2; t += blockDim.x) {
          const int a = ((t & ~(j - 1)) << 1) | (t & (j - 1)), b = a + j;
          const bool up = (a & k) == 0;
          const bool b_first = sp[b] > sp[a] || (sp[b] == sp[a] && kk[b] < kk[a]);
          if (b_first == up) {
            const unsigned long long tp = sp[a], tk = kk[a], ta = aa[a];
            sp[a] = sp[b]; kk[a] = kk[b]; aa[a] = aa[b];
            sp[b] = tp; kk[b] = tk; aa[b] = ta;
          }
        }
        __syncthreads();
      }
    }
    for (int x = threadIdx.x; x < m; x += blockDim.x) {
      Item it;
      it.p = sp[x];
      it.key = kk[x];
      it.aux = aa[x];
      out[x] = it;
    }
  }
  if (threadIdx.x == 0) *gate = 0u;
}

// ---- prefilter for a short K of a longer list -------------------------------
// The bits in which the p of the list differ from the first item's: the
// bits above the highest of them are the same in every item, so the ten bits
// from it downwards are a bin that is monotone in p.  A histogram of those
// bins gives the lowest bin whose count from the top reaches K; a second
// histogram of the next ten bits, over the items of that bin only, refines
// it (values spread over several octaves, such as the bits of doubles,
// leave most items in one first-level bin).  The items above the refined
// threshold (K plus the others of its bin) are compacted for the one-block
// selection.
__global__ void __launch_bounds__(256)
k_pf_diff(const Item* __restrict__ in, unsigned long long n, SelState* st) {
  const unsigned long long v0 = in[0].p;
  unsigned long long diff = 0;
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (unsigned long long)gridDim.x * blockDim.x)
    diff |= in[x].p ^ v0;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) diff |= __shfl_xor_sync(0xFFFFFFFFu, diff, off);
  if ((threadIdx.x & 31) == 0 && diff) atomicOr(&st->maxp, diff);
}

__device__ __forceinline__ int pf_shift(unsigned long long diff) {
  const int hb = diff ? 63 - __clzll((long long)diff) : 0;
  return hb > 9 ? hb - 9 : 0;
}

// Level 1 (bins of p >> sh1 over every item) or level 2 (bins of p >> sh2
// over the items in the level-1 threshold bin).  The last block picks the
// bin where the count from the top reaches K (level 1), or K less the items
// above that bin (level 2); level 1 also leaves that count in st->positive
// and clears the histogram for level 2.
template <int kLevel>
__global__ void __launch_bounds__(256)
k_pf_hist(const Item* __restrict__ in, unsigned long long n, unsigned long long K, SelState* st) {
  __shared__ unsigned int h[1024];
  for (int b = threadIdx.x; b < 1024; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const int sh1 = pf_shift(st->maxp);
  const int sh2 = sh1 > 10 ? sh1 - 10 : 0;
  const unsigned long long theta1 = kLevel == 2 ? st->theta : 0ull;
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long v = in[x].p;
    if (kLevel == 1) atomicAdd(&h[(v >> sh1) & 1023u], 1u);
    else if (((v >> sh1) & 1023u) == theta1) atomicAdd(&h[(v >> sh2) & 1023u], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 1024; b += blockDim.x)
    if (h[b]) atomicAdd(&st->lhist[b], h[b]);
  __threadfence();
  __shared__ unsigned int is_last;
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->ticket3, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const unsigned long long k = kLevel == 1 ? K : K - st->positive;
  unsigned long long total = 0;
  const int b = block_pick_from_top<1024>(st->lhist, k, &total);
  const unsigned long long pick = b >= 0 ? (unsigned long long)b : 0ull;
  if (kLevel == 1) {
    // The items in bins above the pick, then a clear histogram.
    __shared__ unsigned long long above;
    if (threadIdx.x == 0) above = 0;
    __syncthreads();
    unsigned long long mine = 0;
    for (int q = threadIdx.x; q < 1024; q += blockDim.x)
      if ((unsigned long long)q > pick) mine += __ldcg(st->lhist + q);
    atomicAdd(&above, mine);
    __syncthreads();
    for (int q = threadIdx.x; q < 1024; q += blockDim.x) st->lhist[q] = 0;
    if (threadIdx.x == 0) {
      st->theta = pick;
      st->positive = above;
      st->ticket3 = 0;
    }
  } else if (threadIdx.x == 0) {
    st->tp = pick;
  }
}

__global__ void __launch_bounds__(256)
k_pf_compact(const Item* __restrict__ in, unsigned long long n, const SelState* st,
             Item* __restrict__ out, unsigned long long* counter, uint64_t cap) {
  const int sh1 = pf_shift(st->maxp);
  const int sh2 = sh1 > 10 ? sh1 - 10 : 0;
  const unsigned long long theta1 = st->theta, theta2 = st->tp;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long rounds = (n + stride - 1) / stride;
  for (unsigned long long r = 0; r < rounds; ++r) {
    const unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x + r * stride;
    bool want = false;
    Item it;
    if (x < n) {
      it = in[x];
      const unsigned long long b1 = (it.p >> sh1) & 1023u;
      want = b1 > theta1 || (b1 == theta1 && ((it.p >> sh2) & 1023u) >= theta2);
    }
    append_block1(out, counter, want, it, cap);
  }
}

void block_select_dev(mad_ctx* ctx, const Item* in, uint64_t cap, uint64_t K,
                      const unsigned long long* n_dev, bool sorted, Item* tile_sorted,
                      uint32_t* pos, Item* out, unsigned int* gate, unsigned int* over_err,
                      cudaStream_t st) {
  static bool attr = false;
  const size_t smem = (size_t)(kBlockSel + 3 * kBlockSort) * sizeof(unsigned long long);
  if (!attr) {
    cudaFuncSetAttribute(k_block_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  if (sorted && K > (uint64_t)kBlockSort) {   // too many to sort in one block
    tile_select_dev(ctx, in, cap, K, n_dev, over_err, tile_sorted, pos, out, st);
    return;
  }
  k_block_select<<<1, 1024, smem, st>>>(in, cap, n_dev, (unsigned int)K, out, sorted ? 1 : 0,
                                        gate);
  count_launch(ctx);
  tile_select_dev(ctx, in, cap, K, n_dev, over_err, tile_sorted, pos, out, st, gate);
}

size_t dev_select_state_bytes() { return ((sizeof(SelState) + 255) / 256) * 256; }

// The sorted top K (K <= kBlockSort < n <= kTileSortMax) of ws.l0[0..n) into
// ws.out: the prefilter, then the one-block selection of the compacted
// items; when more than kBlockSel of them tie into the threshold bin, the
// tile kernels (gated on the block's word) select from the whole list.
void prefilter_select(mad_ctx* ctx, const SelectWs& ws, uint64_t n, uint64_t K, cudaStream_t st) {
  SelState* dst = (SelState*)ws.state;
  cudaMemsetAsync(dst, 0, sizeof(SelState), st);
  cudaMemsetAsync(ws.counter, 0, sizeof(unsigned long long), st);
  unsigned int* gate = (unsigned int*)(ws.counter + 2);
  const unsigned blocks = grid_for(n, 152 * 4);
  k_pf_diff<<<blocks, 256, 0, st>>>(ws.l0, n, dst);
  k_pf_hist<1><<<blocks, 256, 0, st>>>(ws.l0, n, K, dst);
  k_pf_hist<2><<<blocks, 256, 0, st>>>(ws.l0, n, K, dst);
  k_pf_compact<<<blocks, 256, 0, st>>>(ws.l0, n, dst, ws.l1, ws.counter, ws.cap_n);
  count_launch(ctx, 4);
  // (the fallback's input positions go to ws.l0: the compacted list holds
  // every item it still needs)
  block_select_dev(ctx, ws.l1, n, K, ws.counter, true, ws.l2, (uint32_t*)ws.l0, ws.out, gate,
                   nullptr, st);
}

void select_hash_dev(mad_ctx* ctx, uint64_t K, const unsigned long long* hcap_dev, void* state,
                     unsigned long long* count, Item* list, Item* sorted, uint32_t* pos,
                     Item* out, cudaStream_t st) {
  SelState* dst = (SelState*)state;
  cudaMemsetAsync(dst, 0, sizeof(SelState), st);
  cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  const uint64_t bound = hash_slot_bound(ctx);
  const unsigned blocks = grid_for(bound, 152 * 8);
  // The threshold from one 4-slot group in 16: the sampled count must reach
  // K/16 plus four standard deviations, so the compaction keeps fewer than
  // K items only rarely; then the exact histogram and compaction run.
  constexpr int kLg = 4;
  const double ks = (double)K / (1 << kLg);
  const unsigned long long Ks = (unsigned long long)(ks + 4.0 * sqrt(ks) + 8.0);
  unsigned int* gate = (unsigned int*)(count + 1);
  k_log_hist<<<(blocks + (1u << kLg) - 1) >> kLg, 256, 0, st>>>(ctx->hvals, bound, Ks, dst,
                                                                 hcap_dev, kLg);
  launch_compact_ge(ctx, blocks, st, ctx->hkeys, ctx->hvals, bound, dst, list, kDevSelectCap,
                    count, hcap_dev);
  k_select_check<<<1, 256, 0, st>>>(dst, count, K, gate);
  k_log_hist<<<blocks, 256, 0, st>>>(ctx->hvals, bound, K, dst, hcap_dev, 0, gate);
  launch_compact_ge(ctx, blocks, st, ctx->hkeys, ctx->hvals, bound, dst, list, kDevSelectCap,
                    count, hcap_dev, gate);
  count_launch(ctx, 5);
  block_select_dev(ctx, list, kDevSelectCap, K, count, false, sorted, pos, out,
                   (unsigned int*)(count + 2), &ctx->sc->err, st);
}

// Device-length start of the radix selection: the list holds min(*count,
// cap) items (more than cap: the compaction overflowed, reported); with no
// more than K of them every one is taken (the threshold stays 0).
__global__ void k_radix_init_dev(SelState* st, const unsigned long long* count, uint64_t cap,
                                 unsigned long long K, unsigned int* err) {
  if (threadIdx.x != 0) return;
  const unsigned long long n = *count;
  if (n > cap) atomicOr(err, DERR_SELECT);
  st->n_cur = n < cap ? n : cap;
  st->k_rem = K;
  st->cur = 0;
  st->done = st->n_cur <= K ? 1 : 0;
}

// k_collect over a list of device length min(*count, cap).
__global__ void __launch_bounds__(256)
k_collect_dev(const Item* __restrict__ l0, const unsigned long long* count, uint64_t cap,
              const SelState* st, Item* __restrict__ out, unsigned long long* counter,
              uint64_t out_cap) {
  const unsigned long long n0 = *count, n = n0 < cap ? n0 : cap;
  const unsigned long long tp = st->tp, tk = st->tk;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long rounds = (n + stride - 1) / stride;
  for (unsigned long long r = 0; r < rounds; ++r) {
    const unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x + r * stride;
    bool want = false;
    Item it;
    if (x < n) {
      it = l0[x];
      want = it.p > tp || (it.p == tp && (~it.key) >= tk);
    }
    append_block1(out, counter, want, it, out_cap);
  }
}

void select_hash_dev_long(mad_ctx* ctx, uint64_t K, const unsigned long long* hcap_dev,
                          void* state, unsigned long long* count, Item* list, Item* l1, Item* l2,
                          uint64_t list_cap, Item* topk, Item* sorted, uint32_t* pos, Item* out,
                          cudaStream_t st) {
  SelState* dst = (SelState*)state;
  cudaMemsetAsync(dst, 0, sizeof(SelState), st);
  cudaMemsetAsync(count, 0, 4 * sizeof(unsigned long long), st);
  const uint64_t bound = hash_slot_bound(ctx);
  const unsigned blocks = grid_for(bound, 152 * 8);
  // Exact log-bucket threshold, then every x at or above it.
  k_log_hist<<<blocks, 256, 0, st>>>(ctx->hvals, bound, K, dst, hcap_dev, 0);
  launch_compact_ge(ctx, blocks, st, ctx->hkeys, ctx->hvals, bound, dst, list, list_cap, count,
                    hcap_dev);
  // The K first by (x desc, key asc): MSB radix select over the 8 bytes of
  // x and the 8 of the key, on the device length.
  k_radix_init_dev<<<1, 32, 0, st>>>(dst, count, list_cap, K, &ctx->sc->err);
  const unsigned rb = grid_for(list_cap, 152 * 4);
  constexpr int kDigits = 16;
  for (int q = 0; q < kDigits; ++q) {
    k_radix_hist<<<rb, 256, 0, st>>>(list, l1, l2, dst, q, 8, kDigits - 1);
    k_radix_filter<<<rb, 256, 0, st>>>(list, l1, l2, dst, q, 8, list_cap);
  }
  k_collect_dev<<<grid_for(list_cap, 152 * 8), 256, 0, st>>>(list, count, list_cap, dst, topk,
                                                             count + 1, K);
  count_launch(ctx, 4 + 2 * kDigits);
  // Sorted: the K items at count[1] through the tile sort.
  tile_select_dev(ctx, topk, K, K, count + 1, &ctx->sc->err, sorted, pos, out, st);
}

void items_to_pairs_dev(mad_ctx* ctx, const Item* items, uint64_t cap,
                        const unsigned long long* n_dev, const mad_pair* cand,
                        const double* cvals, mad_pair* out, uint32_t* n_out, cudaStream_t st) {
  k_to_pairs<<<grid_for(cap ? cap : 1, 1u << 30), 256, 0, st>>>(items, cap, cand, cvals, out,
                                                                 n_dev, n_out);
  count_launch(ctx);
}

// Every occupied key with its value (diagnostics).
__global__ void __launch_bounds__(256)
k_export(const unsigned long long* __restrict__ keys, const long long* __restrict__ vals,
         uint64_t cap_max, unsigned long long* __restrict__ ok, long long* __restrict__ ov,
         uint64_t out_cap, unsigned long long* counter, const unsigned long long* cap_dev) {
  const uint64_t cap = dev_len(cap_max, cap_dev);
  for (uint64_t slot = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < cap;
       slot += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = keys[slot];
    if (key == EMPTY_KEY) continue;
    const unsigned long long pos = atomicAdd(counter, 1ull);
    if (pos < out_cap) {
      ok[pos] = key;
      ov[pos] = vals[slot];
    }
  }
}

// Owner rank of a key in a sharded run (a SplitMix64 mix of the key,
// modulo the number of ranks).
__device__ __forceinline__ uint32_t key_owner(unsigned long long key, uint32_t world) {
  return (uint32_t)(mix64(key ^ 0x5851F42D4C957F2Dull) % world);
}

// Occupied slots of X per owner rank (warp-combined atomics).
__global__ void __launch_bounds__(256)
k_owner_count(const unsigned long long* __restrict__ keys, uint64_t cap_max,
              const unsigned long long* cap_dev, uint32_t world, unsigned long long* counts) {
  const uint64_t cap = dev_len(cap_max, cap_dev);
  const uint64_t cap_up = (cap + 31) & ~31ull;
  const unsigned lane = threadIdx.x & 31;
  for (uint64_t slot = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < cap_up;
       slot += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = slot < cap ? keys[slot] : EMPTY_KEY;
    const int o = key == EMPTY_KEY ? -1 : (int)key_owner(key, world);
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, o);
    if (o >= 0 && lane == (unsigned)(__ffs(peers) - 1))
      atomicAdd(&counts[o], (unsigned long long)__popc(peers));
  }
}

// Every occupied slot to its owner's segment [off[o], off[o + 1]).
__global__ void __launch_bounds__(256)
k_owner_scatter(const unsigned long long* __restrict__ keys, const long long* __restrict__ vals,
                uint64_t cap_max, const unsigned long long* cap_dev, uint32_t world,
                const unsigned long long* __restrict__ off, unsigned long long* cursor,
                unsigned long long* __restrict__ ok, long long* __restrict__ ov, uint64_t out_cap) {
  const uint64_t cap = dev_len(cap_max, cap_dev);
  const uint64_t cap_up = (cap + 31) & ~31ull;
  const unsigned lane = threadIdx.x & 31;
  for (uint64_t slot = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < cap_up;
       slot += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = slot < cap ? keys[slot] : EMPTY_KEY;
    const int o = key == EMPTY_KEY ? -1 : (int)key_owner(key, world);
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, o);
    if (o < 0) continue;
    const unsigned leader = __ffs(peers) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&cursor[o], (unsigned long long)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    const unsigned long long pos = off[o] + base + __popc(peers & ((1u << lane) - 1));
    if (pos < out_cap) {
      ok[pos] = key;
      ov[pos] = vals[slot];
    }
  }
}

// Candidate pairs with x > 0 as select items (p = x, aux = position).
__global__ void k_pair_items(const mad_pair* __restrict__ pairs, unsigned long long n,
                             Item* __restrict__ items, unsigned long long* counter) {
  const unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const mad_pair pr = pairs[q];
  if (pr.x <= 0) return;
  Item it;
  it.p = (unsigned long long)pr.x;
  it.key = ((unsigned long long)pr.i << 32) | pr.j;
  it.aux = q;
  items[atomicAdd(counter, 1ull)] = it;
}

__global__ void k_items_to_input_pairs(const Item* __restrict__ items, unsigned long long n,
                                       const mad_pair* __restrict__ pairs,
                                       mad_pair* __restrict__ out) {
  const unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = pairs[items[q].aux];
}

mad_status export_x_by_owner(mad_ctx* ctx, uint32_t world, uint64_t* keys, int64_t* vals,
                             uint64_t cap, uint64_t* offsets_host, cudaStream_t st) {
  // scratch: counts (world), offsets (world + 1), cursors (world)
  unsigned long long* counts = (unsigned long long*)ctx->scratch;
  unsigned long long* off = counts + world;
  unsigned long long* cursor = off + world + 1;
  cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (3 * (size_t)world + 1), st);
  const uint64_t bound = hash_slot_bound(ctx);
  k_owner_count<<<grid_for(bound, 152 * 8), 256, 0, st>>>(ctx->hkeys, bound, hash_extent(ctx),
                                                          world, counts);
  count_launch(ctx);
  std::vector<unsigned long long> hc(world);
  cudaMemcpyAsync(hc.data(), counts, sizeof(unsigned long long) * world, cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  std::vector<unsigned long long> ho(world + 1, 0);
  for (uint32_t o = 0; o < world; ++o) ho[o + 1] = ho[o] + hc[o];
  for (uint32_t o = 0; o <= world; ++o) offsets_host[o] = ho[o];
  if (ho[world] > cap) return MAD_OK;   // the caller sees the total and sizes up
  cudaMemcpyAsync(off, ho.data(), sizeof(unsigned long long) * (world + 1), cudaMemcpyHostToDevice,
                  st);
  k_owner_scatter<<<grid_for(bound, 152 * 8), 256, 0, st>>>(
      ctx->hkeys, ctx->hvals, bound, hash_extent(ctx), world, off, cursor,
      (unsigned long long*)keys, (long long*)vals, cap);
  count_launch(ctx);
  return cuda_status(cudaStreamSynchronize(st));
}

mad_status select_pairs(mad_ctx* ctx, const mad_pair* pairs, uint64_t n, uint64_t K,
                        mad_pair* out, uint64_t* n_sel, cudaStream_t st) {
  *n_sel = 0;
  if (n == 0 || K == 0) return MAD_OK;
  const size_t ws_bytes = (select_ws_bytes(n, K) + 255) & ~(size_t)255;
  mad_status rs = ensure_scratch(ctx, ws_bytes + 256, st);
  if (rs != MAD_OK) return rs;
  const SelectWs ws = select_ws_carve(ctx->scratch, n, K);
  unsigned long long* counter = (unsigned long long*)((char*)ctx->scratch + ws_bytes);
  cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  k_pair_items<<<grid_for(n, 1u << 30), 256, 0, st>>>(pairs, n, ws.l0, counter);
  count_launch(ctx);
  unsigned long long npos = 0;
  cudaMemcpyAsync(&npos, counter, sizeof(npos), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  if ((rs = select_list(ctx, ws, npos, K, 8, n_sel, st)) != MAD_OK) return rs;
  if (*n_sel) {
    k_items_to_input_pairs<<<grid_for(*n_sel, 1u << 30), 256, 0, st>>>(ws.out, *n_sel, pairs, out);
    count_launch(ctx);
  }
  return cuda_status(cudaStreamSynchronize(st));
}

mad_status export_x(mad_ctx* ctx, uint64_t* keys, int64_t* vals, uint64_t cap, uint64_t* n,
                    unsigned long long* counter, cudaStream_t st) {
  cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  k_export<<<grid_for(hash_slot_bound(ctx), 152 * 8), 256, 0, st>>>(ctx->hkeys, ctx->hvals,
                                                                    hash_slot_bound(ctx),
                                                         (unsigned long long*)keys,
                                                         (long long*)vals, cap, counter,
                                                         hash_extent(ctx));
  count_launch(ctx);
  unsigned long long cnt = 0;
  cudaMemcpyAsync(&cnt, counter, sizeof(cnt), cudaMemcpyDeviceToHost, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  *n = cnt;
  return cuda_status(e);
}

}  // namespace mad
