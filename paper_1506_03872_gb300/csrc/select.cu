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

// Warp-aggregated append of `it` when `want`.
__device__ __forceinline__ void append(Item* out, unsigned long long* counter, bool want,
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
    append(out, &st->n_next, want, it, cap);
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
    append(out, counter, want, it, cap);
  }
}

// ---- hash path: one-pass log-bucket histogram, then a threshold compaction --
// Bucket of v >= 1: 16 * floor(log2 v) + the 4 bits below the leading bit
// (1024 buckets, monotone in v).  The collect threshold is the lower bound
// of the bucket in which the count from the top reaches K, so at least K
// items (all of the top K) pass and few more do.
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

__global__ void __launch_bounds__(256)
k_log_hist(const long long* __restrict__ vals, uint64_t cap, unsigned long long K,
           SelState* st) {
  __shared__ unsigned int h[1024];
  for (int b = threadIdx.x; b < 1024; b += blockDim.x) h[b] = 0;
  __syncthreads();
  unsigned long long mx = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t rounds = (cap + stride - 1) / stride;
  for (uint64_t r = 0; r < rounds; ++r) {
    const uint64_t slot = r * stride + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const long long v = slot < cap ? vals[slot] : 0;
    const uint32_t bin = v > 0 ? log_bucket((unsigned long long)v) : 0xFFFFu;
    // one shared-memory atomic per distinct bucket per warp
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, bin);
    if (v > 0) {
      if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[bin], __popc(peers));
      if ((unsigned long long)v > mx) mx = (unsigned long long)v;
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
  if (!is_last || threadIdx.x != 0) return;
  __threadfence();
  volatile unsigned int* gh = st->lhist;
  unsigned long long cum = 0, theta = 1;  // fewer than K positive: take all
  for (int b = 1023; b >= 0; --b) {
    cum += gh[b];
    if (cum >= K) {
      theta = bucket_floor((uint32_t)b);
      break;
    }
  }
  unsigned long long total = 0;
  for (int b = 0; b < 1024; ++b) total += gh[b];
  st->theta = theta;
  st->positive = total;
}

__global__ void __launch_bounds__(256)
k_compact_ge(const unsigned long long* __restrict__ keys, const long long* __restrict__ vals,
             uint64_t cap, const SelState* st, Item* __restrict__ out, uint64_t out_cap,
             unsigned long long* counter) {
  const unsigned long long theta = st->theta;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t rounds = (cap + stride - 1) / stride;
  const uint64_t start = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (uint64_t r = 0; r < rounds; ++r) {
    const uint64_t slot = start + r * stride;
    bool want = false;
    Item it;
    if (slot < cap) {
      const long long v = vals[slot];
      if (v > 0 && (unsigned long long)v >= theta) {
        it.p = (unsigned long long)v;
        it.key = keys[slot];
        it.aux = slot;
        want = true;
      }
    }
    append(out, counter, want, it, out_cap);
  }
}

// ---- single-block MSB radix select for short lists -------------------------
constexpr unsigned kBlockSelectMax = 1u << 15;

__global__ void __launch_bounds__(1024)
k_select_block(const Item* __restrict__ list, unsigned n, unsigned K, int dp,
               Item* __restrict__ out) {
  __shared__ unsigned int h[256];
  __shared__ unsigned long long s_tp, s_tk, s_mp, s_mk;
  __shared__ unsigned int s_krem, s_count;
  __shared__ int s_done;
  if (threadIdx.x == 0) {
    s_tp = s_tk = s_mp = s_mk = 0;
    s_krem = K;
    s_done = 0;
    s_count = 0;
  }
  __syncthreads();
  const int last_q = dp + 7;
  for (int q = 0; q <= last_q; ++q) {
    if (s_done) break;
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const unsigned long long tp = s_tp, tk = s_tk, mp = s_mp, mk = s_mk;
    for (unsigned x = threadIdx.x; x < n; x += blockDim.x) {
      const Item it = list[x];
      if ((it.p & mp) == tp && ((~it.key) & mk) == tk) atomicAdd(&h[digit_of(it, q, dp)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned above = 0;
      int b = 255;
      for (; b > 0; --b) {
        if (above + h[b] >= s_krem) break;
        above += h[b];
      }
      s_krem -= above;
      if (q < dp) {
        const int sh = 8 * (dp - 1 - q);
        s_tp |= (unsigned long long)b << sh;
        s_mp |= 0xFFull << sh;
      } else {
        const int sh = 8 * (7 - (q - dp));
        s_tk |= (unsigned long long)b << sh;
        s_mk |= 0xFFull << sh;
      }
      if (h[b] == s_krem || q == last_q) s_done = 1;
    }
    __syncthreads();
  }
  const unsigned long long tp = s_tp, tk = s_tk;
  for (unsigned x = threadIdx.x; x < n; x += blockDim.x) {
    const Item it = list[x];
    if (it.p > tp || (it.p == tp && (~it.key) >= tk)) {
      const unsigned pos = atomicAdd(&s_count, 1u);
      if (pos < K) out[pos] = it;
    }
  }
}

// ---- rank sort for short lists ---------------------------------------------
// Item x lands at its rank: the number of items that come before it by
// (p desc, key asc, position asc).  The position makes ranks a permutation
// even for repeated keys; only the first K ranks are written.  The n^2
// comparisons are split over blockIdx.y slices of the list, each slice adding
// its count with one atomic per item, so a list of a few thousand items still
// spreads over the whole GPU.
constexpr unsigned kRankSortMax = 1u << 14;
constexpr int kRankTile = 1024;

__global__ void __launch_bounds__(256)
k_rank_count(const Item* __restrict__ in, unsigned n, unsigned slice, unsigned* __restrict__ rank) {
  __shared__ ulonglong2 sv[kRankTile];
  const unsigned x = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lo = blockIdx.y * slice;
  const unsigned hi = min(n, lo + slice);
  unsigned long long mp = 0, mk = 0;
  if (x < n) {
    mp = in[x].p;
    mk = in[x].key;
  }
  unsigned cnt = 0;
  for (unsigned base = lo; base < hi; base += kRankTile) {
    const unsigned len = min((unsigned)kRankTile, hi - base);
    __syncthreads();
    for (unsigned q = threadIdx.x; q < len; q += blockDim.x)
      sv[q] = make_ulonglong2(in[base + q].p, in[base + q].key);
    __syncthreads();
    if (x < n) {
#pragma unroll 8
      for (unsigned q = 0; q < len; ++q) {
        const ulonglong2 o = sv[q];
        const bool before = o.x > mp || (o.x == mp && (o.y < mk || (o.y == mk && base + q < x)));
        cnt += before ? 1u : 0u;
      }
    }
  }
  if (x < n && cnt) atomicAdd(&rank[x], cnt);
}

__global__ void __launch_bounds__(256)
k_rank_scatter(const Item* __restrict__ in, unsigned n, unsigned K, const unsigned* __restrict__ rank,
               Item* __restrict__ out) {
  const unsigned x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < n) {
    const unsigned r = rank[x];
    if (r < K) out[r] = in[x];
  }
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

__global__ void k_to_pairs(const Item* __restrict__ items, unsigned long long n,
                           const mad_pair* __restrict__ cand, const double* __restrict__ cvals,
                           mad_pair* __restrict__ out) {
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
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

mad_status select_list(mad_ctx* ctx, const SelectWs& ws, uint64_t n, uint64_t K, int dp,
                       uint64_t* n_sel, cudaStream_t st) {
  const uint64_t take = K < n ? K : n;
  *n_sel = take;
  if (take == 0) return MAD_OK;
  unsigned long long n2 = 0;
  // Short lists are ranked whole (ranks >= K are dropped).  Longer ones
  // first pick the K largest, unordered, into `sel`; those are then ranked
  // when K is short, else sorted in place by a bitonic network.
  const bool rank_sort = take <= kRankSortMax;
  Item* sel = rank_sort ? ws.l2 : ws.out;
  uint64_t nr = take;   // items ranked
  if (take == n || n <= kRankSortMax) {
    sel = ws.l0;
    nr = n;
    if (!rank_sort) cudaMemcpyAsync(ws.out, ws.l0, n * sizeof(Item), cudaMemcpyDeviceToDevice, st);
  } else if (n <= kBlockSelectMax) {
    k_select_block<<<1, 1024, 0, st>>>(ws.l0, (unsigned)n, (unsigned)K, dp, sel);
    count_launch(ctx);
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
    // The filter passes ping-pong through l1/l2; collect from l0 with the
    // final digit state, so `sel` may reuse l2 once they are done.
    cudaMemsetAsync(ws.counter, 0, sizeof(unsigned long long), st);
    k_collect<<<grid_for(n, 152 * 8), 256, 0, st>>>(ws.l0, n, dst, sel, ws.counter,
                                                     rank_sort ? ws.cap_n : ws.cap_out);
    count_launch(ctx);
  }
  if (rank_sort) {
    unsigned* rank = (unsigned*)ws.l1;
    const unsigned nt = (unsigned)nr;
    const unsigned nb = (nt + 255) / 256;
    unsigned slices = std::min((152u * 8u + nb - 1) / nb, nb);
    const unsigned slice = (nt + slices - 1) / slices;
    slices = (nt + slice - 1) / slice;
    cudaMemsetAsync(rank, 0, nt * sizeof(unsigned), st);
    k_rank_count<<<dim3(nb, slices), 256, 0, st>>>(sel, nt, slice, rank);
    k_rank_scatter<<<nb, 256, 0, st>>>(sel, nt, (unsigned)take, rank, ws.out);
    count_launch(ctx, 2);
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
  const unsigned blocks = grid_for(ctx->hcap, 152 * 8);
  k_log_hist<<<blocks, 256, 0, st>>>(ctx->hvals, ctx->hcap, K, dst);
  k_compact_ge<<<blocks, 256, 0, st>>>(ctx->hkeys, ctx->hvals, ctx->hcap, dst, ws.l0, ws.cap_n,
                                       ws.counter);
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
  k_to_pairs<<<grid_for(n, 1u << 30), 256, 0, st>>>(items, n, cand, cvals, out);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

// Every occupied key with its value (diagnostics).
__global__ void __launch_bounds__(256)
k_export(const unsigned long long* __restrict__ keys, const long long* __restrict__ vals,
         uint64_t cap, unsigned long long* __restrict__ ok, long long* __restrict__ ov,
         uint64_t out_cap, unsigned long long* counter) {
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

mad_status export_x(mad_ctx* ctx, uint64_t* keys, int64_t* vals, uint64_t cap, uint64_t* n,
                    unsigned long long* counter, cudaStream_t st) {
  cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  k_export<<<grid_for(ctx->hcap, 152 * 8), 256, 0, st>>>(ctx->hkeys, ctx->hvals, ctx->hcap,
                                                         (unsigned long long*)keys,
                                                         (long long*)vals, cap, counter);
  count_launch(ctx);
  unsigned long long cnt = 0;
  cudaMemcpyAsync(&cnt, counter, sizeof(cnt), cudaMemcpyDeviceToHost, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  *n = cnt;
  return cuda_status(e);
}

}  // namespace mad
