// Exact comparator for 0/1 inputs: the t largest c_ij of C = A B by direct
// sparse computation (the paper's exact computation for comparison, Sec.
// 4.3, which forms C one sparse vector at a time and keeps the top entries
// in a priority queue), rebuilt for the GPU around a fused threshold.
//
// For 0/1 inputs c_ij counts the k with a_ik = b_kj = 1, so c_ij <=
// min(nnz(a_i*), nnz(b_*j)).  With theta a lower bound on the t-th largest
// entry tau, no row with fewer than theta entries and no column of B with
// fewer than theta entries can hold a pair of the top t, so:
//
//   1. pilot: the exact counts among the ~2048 rows of A and columns of B of
//      largest degree; the t-th largest of them is such a theta (t entries
//      of C are at least that large);
//   2. main pass over the rows with nnz >= theta against the columns with
//      nnz >= theta only: B is filtered to those columns and relabelled by
//      their rank (a monotone map, so every row of B stays sorted), each row
//      i of C is accumulated in shared-memory count windows (one block per
//      row, rows handed out through an atomic counter in decreasing degree
//      order), and its entries with c >= theta go to a candidate list;
//   3. the t largest candidates by (c desc, key asc), sorted.
//
// Entries equal to the t-th value are ties; if the candidates overflow the
// list, the exact tau comes from the histogram of the emitted counts and
// the pass repeats: every c > tau, then the smallest keys among c == tau
// (per-row tie counts, their prefix over rows in index order, and the first
// ties of the boundary row in ascending j).  The result equals the oracle's
// row-wise sparse product for any input.  With MAD_SPARSE_NO_BOUND the main
// pass takes every row and column (only the threshold filters entries).
#include <cuda_runtime.h>
#include <stdint.h>

#include "mad_internal.cuh"

namespace mad {
namespace {

constexpr int kSpBlock = 256;
constexpr int kSpWarps = kSpBlock / 32;
constexpr uint32_t kSpWindowMax = 24576;       // labels per shared window (96 KB)
constexpr uint32_t kPilot = 2048;              // rows and columns of the pilot
constexpr uint32_t kHistSmem = 4096;           // pilot histogram bins (clamped)
constexpr uint32_t kHistGlobal = 65536;        // main-pass histogram bins (clamped)
constexpr uint64_t kSpListCap = 1ull << 20;    // candidate list entries
constexpr unsigned FULL = 0xffffffffu;

struct SpScalars {
  unsigned int bins[2][32];        // log2-degree bucket counts (rows, columns)
  unsigned int cur[2][32];         // scatter cursors
  unsigned long long count;        // candidates emitted (may pass the capacity)
  unsigned int row_next;           // persistent row counter
  unsigned int theta;              // threshold read from a histogram
  unsigned int row_lim, lim_x;     // tie-limited emission
  unsigned long long need;         // ties still to take
  unsigned int err;
  unsigned int pad;
};

__device__ __forceinline__ uint32_t deg_of(const int64_t* ptr, const uint32_t* cnt, uint64_t i) {
  return ptr ? (uint32_t)(ptr[i + 1] - ptr[i]) : cnt[i];
}

// Column counts of B: cb[j] = nnz of column j.
__global__ void k_col_counts(const int32_t* __restrict__ col, uint64_t nnz, uint32_t* cb) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&cb[col[e]], 1u);
}

// Row degrees as counts (Gram inputs: the columns of B = A^T are the rows
// of A).
__global__ void k_row_degrees(const int64_t* __restrict__ ptr, uint64_t n, uint32_t* out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)(ptr[i + 1] - ptr[i]);
}

// Indices with degree >= th, counted per floor(log2(degree)) bucket.
__global__ void k_logbin_count(const int64_t* ptr, const uint32_t* cnt, uint64_t n, uint32_t th,
                               unsigned int* bins) {
  __shared__ unsigned int sb[32];
  if (threadIdx.x < 32) sb[threadIdx.x] = 0;
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t dg = deg_of(ptr, cnt, i);
    if (dg >= th && dg > 0) atomicAdd(&sb[31 - __clz(dg)], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 32 && sb[threadIdx.x]) atomicAdd(&bins[threadIdx.x], sb[threadIdx.x]);
}

// The same indices in decreasing bucket order (any order within a bucket):
// a schedule and a choice of the heaviest rows, not a result.
__global__ void k_logbin_scatter(const int64_t* ptr, const uint32_t* cnt, uint64_t n, uint32_t th,
                                 const unsigned int* bins, unsigned int* cur, uint32_t* order) {
  __shared__ unsigned int off[32];
  if (threadIdx.x < 32) {
    unsigned int s = 0;
    for (int b = 31; b > (int)threadIdx.x; --b) s += bins[b];
    off[threadIdx.x] = s;
  }
  __syncthreads();
  const unsigned lane = threadIdx.x & 31;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t n_up = (n + 31) & ~31ull;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_up; i += stride) {
    const uint32_t dg = i < n ? deg_of(ptr, cnt, i) : 0;
    const bool take = i < n && dg >= th && dg > 0;
    const int b = take ? 31 - __clz(dg) : -1;
    const unsigned peers = __match_any_sync(FULL, b);
    if (take) {
      const unsigned leader = __ffs(peers) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(&cur[b], (unsigned)__popc(peers));
      base = __shfl_sync(peers, base, leader);
      order[off[b] + base + __popc(peers & ((1u << lane) - 1))] = (uint32_t)i;
    }
  }
}

__global__ void k_mark_list(const uint32_t* __restrict__ list, uint32_t h, uint32_t* sel) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < h) sel[list[q]] = 1u;
}

__global__ void k_mark_deg(const uint32_t* __restrict__ cb, uint64_t n, uint32_t th, uint32_t* sel) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (uint64_t)gridDim.x * blockDim.x)
    sel[j] = (cb[j] >= th && cb[j] > 0) ? 1u : 0u;
}

__global__ void k_colmap(const uint32_t* __restrict__ sel, const uint32_t* __restrict__ pre,
                         uint64_t n, uint32_t* colmap) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (uint64_t)gridDim.x * blockDim.x)
    if (sel[j]) colmap[pre[j]] = (uint32_t)j;
}

// Entries of each row of B whose column is selected (one warp per row).
__global__ void k_bf_count(const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                           uint64_t d, const uint32_t* __restrict__ sel, uint32_t* len) {
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned lane = threadIdx.x & 31;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t k = warp; k < d; k += nw) {
    const int64_t e0 = bptr[k], e1 = bptr[k + 1];
    unsigned c = 0;
    for (int64_t e = e0 + lane; e < e1; e += 32) c += sel[bcol[e]];
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if (lane == 0) len[k] = c;
  }
}

// The selected entries, relabelled by their column's rank, in order.
__global__ void k_bf_fill(const int64_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
                          uint64_t d, const uint32_t* __restrict__ sel,
                          const uint32_t* __restrict__ pre, const uint32_t* __restrict__ optr,
                          uint32_t* ocol) {
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned lane = threadIdx.x & 31;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t k = warp; k < d; k += nw) {
    const int64_t e0 = bptr[k], e1 = bptr[k + 1];
    uint32_t out = optr[k];
    for (int64_t base = e0; base < e1; base += 32) {
      const int64_t e = base + lane;
      uint32_t j = 0, s = 0;
      if (e < e1) {
        j = (uint32_t)bcol[e];
        s = sel[j];
      }
      const unsigned bal = __ballot_sync(FULL, s != 0);
      if (s) ocol[out + __popc(bal & ((1u << lane) - 1))] = pre[j];
      out += __popc(bal);
    }
  }
}

// First position in [lo, hi) whose label is >= L (hi if none); labels
// ascending.  All lanes of the warp call it with the same arguments.
__device__ __forceinline__ uint32_t warp_lower_bound(const uint32_t* __restrict__ lab,
                                                     uint32_t lo, uint32_t hi, uint32_t L,
                                                     unsigned lane) {
  while (hi - lo > 32) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t pos = lo + lane * step;
    const uint32_t v = pos < hi ? lab[pos] : 0xffffffffu;
    const unsigned c = __popc(__ballot_sync(FULL, v < L));
    if (c == 0) return lo;
    const uint32_t nlo = lo + (c - 1) * step + 1;
    const uint32_t nhi = lo + c * step < hi ? lo + c * step : hi;
    lo = nlo;
    hi = nhi;
  }
  const uint32_t pos = lo + lane;
  const uint32_t v = pos < hi ? lab[pos] : 0xffffffffu;
  return lo + __popc(__ballot_sync(FULL, v < L));
}

struct SpRowParams {
  const int64_t* aptr;
  const int32_t* acol;
  const uint32_t* rows;           // schedule of rows
  const unsigned int* nrows_bins; // number of rows: sum of these 32 bucket counts
  uint32_t nrows_cap;             // the schedule never holds more than this
  const uint32_t* bptr;           // filtered B: row k's labels at [bptr[k], bptr[k+1])
  const uint32_t* bcol;
  uint32_t nlab;                  // selected columns
  const uint32_t* sel;            // column selected (n)
  const uint32_t* pre;            // rank of column j among the selected (n + 1)
  const uint32_t* colmap;         // label -> column
  int gram, excl;
  uint32_t window;                // labels per shared window
  uint32_t th_emit;               // emit every c >= th_emit (0xffffffff: none)
  uint32_t th_tie;                // tie value (tie_mode > 0)
  int tie_mode;                   // 0 off, 1 count ties per row, 2 emit ties under the limit
  unsigned long long* tiecnt;     // per-row tie counts (tie_mode 1)
  int hist_smem;                  // histogram of emitted c in shared memory (kHistSmem bins)
  unsigned int* hist;             // clamped histogram of emitted c (null: none)
  uint32_t hist_bins;
  Item* list;
  unsigned long long cap;
  SpScalars* sc;
};

// One block per row of C at a time: row i = sum over k in row i of A of row
// k of the filtered B, counted in shared memory one window of labels at a
// time; the window's entries are tested against the threshold and cleared
// while they are read.  Gram inputs count unordered pairs: labels from the
// rank of column i on (past it when the diagonal is excluded).
__global__ void __launch_bounds__(kSpBlock) k_spgemm_rowblock_topk(SpRowParams p) {
  extern __shared__ uint32_t smem[];
  uint32_t* acc = smem;                       // p.window counts
  uint32_t* shist = smem + p.window;          // kHistSmem bins when p.hist_smem
  __shared__ unsigned int s_row;
  __shared__ unsigned int s_wsum[kSpWarps];
  __shared__ unsigned long long s_run;
  __shared__ unsigned long long s_ties;
  const unsigned tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (uint32_t q = tid; q < p.window; q += kSpBlock) acc[q] = 0;
  if (p.hist_smem)
    for (uint32_t q = tid; q < kHistSmem; q += kSpBlock) shist[q] = 0;
  unsigned nrows = 0;
  for (int b = 0; b < 32; ++b) nrows += p.nrows_bins[b];
  if (nrows > p.nrows_cap) nrows = p.nrows_cap;
  const uint32_t row_lim = p.tie_mode == 2 ? p.sc->row_lim : 0;
  const uint32_t lim_x = p.tie_mode == 2 ? p.sc->lim_x : 0;
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s_row = atomicAdd(&p.sc->row_next, 1u);
      s_run = 0;
      s_ties = 0;
    }
    __syncthreads();
    const unsigned qr = s_row;
    if (qr >= nrows) break;
    const uint32_t i = p.rows[qr];
    if (p.tie_mode == 2 && i > row_lim) continue;
    const int64_t a0 = p.aptr[i], a1 = p.aptr[i + 1];
    uint32_t lo = 0;
    if (p.gram) lo = p.pre[i] + (p.excl ? p.sel[i] : 0u);
    const bool limited = p.tie_mode == 2 && i == row_lim;
    for (uint32_t w0 = (lo / p.window) * p.window; w0 < p.nlab; w0 += p.window) {
      const uint32_t w1 = w0 + p.window < p.nlab ? w0 + p.window : p.nlab;
      const uint32_t L = lo > w0 ? lo : w0;
      // Accumulate: warp per entry a_ik, lanes over row k of the filtered B.
      for (int64_t q = a0 + warp; q < a1; q += kSpWarps) {
        const uint32_t k = (uint32_t)p.acol[q];
        const uint32_t b0 = p.bptr[k], b1 = p.bptr[k + 1];
        if (b0 == b1) continue;
        const uint32_t start = L == 0 ? b0 : warp_lower_bound(p.bcol, b0, b1, L, lane);
        for (uint32_t e = start + lane; e < b1; e += 32) {
          const uint32_t lab = p.bcol[e];
          if (lab >= w1) break;
          atomicAdd(&acc[lab - w0], 1u);
        }
      }
      __syncthreads();
      // Scan the window: threshold, emit, clear.
      for (uint32_t base = L; base < w1; base += kSpBlock) {
        const uint32_t q = base + tid;
        uint32_t c = 0;
        if (q < w1) {
          c = acc[q - w0];
          if (c) acc[q - w0] = 0;
        }
        uint32_t j = 0;
        bool em = false, tie = false;
        if (c) {
          j = p.colmap[q];
          const bool diag_out = p.excl && !p.gram && j == i;
          em = !diag_out && c >= p.th_emit;
          tie = !diag_out && p.tie_mode != 0 && c == p.th_tie;
        }
        if (p.tie_mode == 1) {
          const unsigned nt = __popc(__ballot_sync(FULL, tie));
          if (lane == 0 && nt) atomicAdd(&s_ties, (unsigned long long)nt);
        } else if (p.tie_mode == 2) {
          if (limited) {
            // rank of this tie among the row's ties in ascending j
            const unsigned bal = __ballot_sync(FULL, tie);
            if (lane == 0) s_wsum[warp] = __popc(bal);
            __syncthreads();
            unsigned before = 0, total = 0;
            for (int w = 0; w < kSpWarps; ++w) {
              if (w < (int)warp) before += s_wsum[w];
              total += s_wsum[w];
            }
            const unsigned long long rank =
                s_run + before + __popc(bal & ((1u << lane) - 1));
            em = tie && rank < lim_x;
            __syncthreads();
            if (tid == 0) s_run += total;
          } else {
            em = tie;   // a row before the boundary row: all its ties
          }
        }
        const unsigned bal = __ballot_sync(FULL, em);
        if (bal) {
          const unsigned leader = __ffs(bal) - 1;
          unsigned long long pos0 = 0;
          if (lane == leader) pos0 = atomicAdd(&p.sc->count, (unsigned long long)__popc(bal));
          pos0 = __shfl_sync(FULL, pos0, leader);
          if (em) {
            const unsigned long long pos = pos0 + __popc(bal & ((1u << lane) - 1));
            if (pos < p.cap) {
              Item it;
              it.p = c;
              it.key = ((unsigned long long)i << 32) | j;
              it.aux = 0;
              p.list[pos] = it;
            }
            if (p.hist_smem)
              atomicAdd(&shist[c < kHistSmem ? c : kHistSmem - 1], 1u);
            else if (p.hist)
              atomicAdd(&p.hist[c < p.hist_bins ? c : p.hist_bins - 1], 1u);
          }
        }
      }
      __syncthreads();
    }
    if (p.tie_mode == 1 && tid == 0 && s_ties) p.tiecnt[i] += s_ties;   // one block per row
  }
  if (p.hist_smem) {
    __syncthreads();
    for (uint32_t q = tid; q < kHistSmem; q += kSpBlock)
      if (shist[q]) atomicAdd(&p.hist[q], shist[q]);
  }
}

// theta = the largest v >= 1 such that at least t emitted counts are >= v
// (the top bin holds every count at or above it), or 1 when fewer than t
// counts were emitted.
__global__ void __launch_bounds__(1024) k_hist_theta(const unsigned int* __restrict__ hist,
                                                     uint32_t nb, unsigned long long t,
                                                     SpScalars* sc) {
  __shared__ unsigned long long s_run;
  __shared__ unsigned long long s_w[32];
  __shared__ int s_found;
  const unsigned tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_run = 0;
    s_found = -1;
  }
  __syncthreads();
  for (int hi = (int)nb; hi > 1; hi -= 1024) {
    const int v = hi - 1 - (int)tid;     // thread tid takes bin v, descending
    unsigned long long h = v >= 1 ? hist[v] : 0;
    unsigned long long x = h;           // inclusive prefix over tid
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(FULL, x, o);
      if ((int)lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    unsigned long long before = 0;
    for (int w = 0; w < (int)warp; ++w) before += s_w[w];
    const unsigned long long ge = s_run + before + x;   // counts >= v
    if (v >= 1 && ge >= t) atomicMax(&s_found, v);
    __syncthreads();
    if (s_found >= 1) break;
    if (tid == 1023) s_run = s_run + before + x;
    __syncthreads();
  }
  if (tid == 0) sc->theta = s_found >= 1 ? (unsigned)s_found : 1u;
}

// Boundary of the tie-limited emission: row_lim is the row in whose ties
// the need runs out (prefix over rows in index order), lim_x the number of
// its ties to take.
__global__ void k_tie_limit(const unsigned long long* __restrict__ tiepre, uint64_t m,
                            unsigned long long t, SpScalars* sc) {
  const unsigned long long have = sc->count;
  const unsigned long long need = t > have ? t - have : 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    if (tiepre[i] < need && need <= tiepre[i + 1]) {
      sc->row_lim = (uint32_t)i;
      sc->lim_x = (uint32_t)(need - tiepre[i]);
      sc->need = need;
    }
  }
}

__global__ void k_sp_to_pairs(const Item* __restrict__ items, uint64_t n, mad_pair* out) {
  const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const Item it = items[q];
  mad_pair pr;
  pr.i = (uint32_t)(it.key >> 32);
  pr.j = (uint32_t)it.key;
  pr.x = 0;
  pr.c = (double)it.p;
  out[q] = pr;
}

unsigned blocks_for(uint64_t n, unsigned cap) {
  const uint64_t b = (n + 255) / 256;
  return (unsigned)(b == 0 ? 1 : (b < cap ? b : cap));
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch of one call.
struct SpWs {
  uint32_t *cb, *rorder, *corder, *sel, *pre, *colmap, *blen, *bp, *bcol, *part, *hist;
  unsigned long long *tiecnt, *tiepre, *part64;
  SpScalars* sc;
  SelectWs sel_ws;
};

size_t sp_ws_bytes(uint64_t m, uint64_t d, uint64_t n, uint64_t nnzb, uint64_t t, SpWs* ws,
                   char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  const uint64_t parts = scan_partial_elems((n > d ? n : d) + 1);
  SpWs w{};
  w.cb = (uint32_t*)take(4 * n);
  w.rorder = (uint32_t*)take(4 * m);
  w.corder = (uint32_t*)take(4 * n);
  w.sel = (uint32_t*)take(4 * (n + 1));
  w.pre = (uint32_t*)take(4 * (n + 1));
  w.colmap = (uint32_t*)take(4 * n);
  w.blen = (uint32_t*)take(4 * (d + 1));
  w.bp = (uint32_t*)take(4 * (d + 1));
  w.bcol = (uint32_t*)take(4 * (nnzb ? nnzb : 1));
  w.part = (uint32_t*)take(4 * parts);
  w.hist = (uint32_t*)take(4 * kHistGlobal);
  w.tiecnt = (unsigned long long*)take(8 * (m + 1));
  w.tiepre = (unsigned long long*)take(8 * (m + 1));
  w.part64 = (unsigned long long*)take(8 * scan_partial_elems(m + 1));
  w.sc = (SpScalars*)take(sizeof(SpScalars));
  char* sb = take(select_ws_bytes(kSpListCap, t));
  if (base) w.sel_ws = select_ws_carve(sb, kSpListCap, t);
  if (ws) *ws = w;
  return off;
}

}  // namespace
}  // namespace mad

using namespace mad;

mad_status mad_sparse_topt(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B, uint32_t t,
                           uint32_t options, mad_pair* out_dev, uint32_t* n_out_host,
                           mad_stream stream) {
  if (!ctx || !A || !B || !out_dev || !n_out_host || t == 0) return MAD_ERR_ARG;
  *n_out_host = 0;
  if (options & ~(uint32_t)MAD_SPARSE_NO_BOUND) return MAD_ERR_ARG;
  if (A->fmt != MAD_CSR || B->fmt != MAD_CSR || A->dt != MAD_BINARY || B->dt != MAD_BINARY)
    return MAD_ERR_UNSUPPORTED;
  if (!A->rowptr || !A->colidx || !B->rowptr || !B->colidx || A->rows <= 0 || A->cols <= 0 ||
      B->cols <= 0)
    return MAD_ERR_ARG;
  if (B->rows != A->cols || A->rows >= (1ll << 31) || B->cols >= (1ll << 31) ||
      A->cols >= (1ll << 31))
    return MAD_ERR_ARG;
  if (t > kSpListCap / 2) return MAD_ERR_UNSUPPORTED;
  const bool gram = (ctx->flags & MAD_GRAM) != 0;
  const bool excl = (ctx->flags & MAD_EXCLUDE_DIAG) != 0;
  if (gram && A->rows != B->cols) return MAD_ERR_ARG;
  const bool bound = !(options & MAD_SPARSE_NO_BOUND);
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t m = (uint64_t)A->rows, d = (uint64_t)A->cols, n = (uint64_t)B->cols;

  int64_t nnz_h[2] = {0, 0};
  cudaMemcpyAsync(&nnz_h[0], A->rowptr + m, 8, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&nnz_h[1], B->rowptr + d, 8, cudaMemcpyDeviceToHost, st);
  cudaError_t ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_status(ce);
  if (nnz_h[0] < 0 || nnz_h[1] < 0 || nnz_h[1] >= (1ll << 31)) return MAD_ERR_ARG;
  const uint64_t nnzb = (uint64_t)nnz_h[1];

  mad_status rs = ensure_scratch(ctx, sp_ws_bytes(m, d, n, nnzb, t, nullptr, nullptr), st);
  if (rs != MAD_OK) return rs;
  SpWs w{};
  sp_ws_bytes(m, d, n, nnzb, t, &w, (char*)ctx->scratch);

  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid_stream = (unsigned)(sms * 8);

  // Column counts and degree orders of rows and columns.
  cudaMemsetAsync(w.sc, 0, sizeof(SpScalars), st);
  if (gram) {
    k_row_degrees<<<blocks_for(n, grid_stream), 256, 0, st>>>(A->rowptr, n, w.cb);
  } else {
    cudaMemsetAsync(w.cb, 0, 4 * n, st);
    k_col_counts<<<blocks_for(nnzb, grid_stream), 256, 0, st>>>(B->colidx, nnzb, w.cb);
  }
  k_logbin_count<<<blocks_for(m, grid_stream), 256, 0, st>>>(A->rowptr, nullptr, m, 1u,
                                                            w.sc->bins[0]);
  k_logbin_count<<<blocks_for(n, grid_stream), 256, 0, st>>>(nullptr, w.cb, n, 1u,
                                                            w.sc->bins[1]);
  k_logbin_scatter<<<blocks_for(m, grid_stream), 256, 0, st>>>(A->rowptr, nullptr, m, 1u,
                                                              w.sc->bins[0], w.sc->cur[0],
                                                              w.rorder);
  k_logbin_scatter<<<blocks_for(n, grid_stream), 256, 0, st>>>(nullptr, w.cb, n, 1u,
                                                              w.sc->bins[1], w.sc->cur[1],
                                                              w.corder);
  count_launch(ctx, 5);
  SpScalars hs{};
  cudaMemcpyAsync(&hs, w.sc, sizeof(SpScalars), cudaMemcpyDeviceToHost, st);
  if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(ce);
  uint64_t rows_nz = 0, cols_nz = 0;
  for (int b = 0; b < 32; ++b) {
    rows_nz += hs.bins[0][b];
    cols_nz += hs.bins[1][b];
  }
  if (rows_nz == 0 || cols_nz == 0) return MAD_OK;   // C = 0: no stored entry

  const size_t smem_max = (size_t)kSpWindowMax * 4 + (size_t)kHistSmem * 4;
  cudaFuncSetAttribute(k_spgemm_rowblock_topk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem_max);

  // Selected columns -> labels and the filtered, relabelled B.
  auto select_columns = [&](bool from_list, uint32_t h, uint32_t th) -> mad_status {
    if (from_list) {
      cudaMemsetAsync(w.sel, 0, 4 * n, st);
      k_mark_list<<<blocks_for(h, 1u << 30), 256, 0, st>>>(w.corder, h, w.sel);
    } else {
      k_mark_deg<<<blocks_for(n, grid_stream), 256, 0, st>>>(w.cb, n, th, w.sel);
    }
    count_launch(ctx);
    mad_status r = scan_exclusive_u32(ctx, w.sel, w.pre, n, w.part, st);
    if (r != MAD_OK) return r;
    k_colmap<<<blocks_for(n, grid_stream), 256, 0, st>>>(w.sel, w.pre, n, w.colmap);
    const unsigned wg = blocks_for(d * 32, (unsigned)sms * 16);
    k_bf_count<<<wg, 256, 0, st>>>(B->rowptr, B->colidx, d, w.sel, w.blen);
    count_launch(ctx, 2);
    if ((r = scan_exclusive_u32(ctx, w.blen, w.bp, d, w.part, st)) != MAD_OK) return r;
    k_bf_fill<<<wg, 256, 0, st>>>(B->rowptr, B->colidx, d, w.sel, w.pre, w.bp, w.bcol);
    count_launch(ctx);
    return cuda_status(cudaGetLastError());
  };

  auto run_rows = [&](uint32_t nlab, const unsigned int* bins, uint32_t rows_cap,
                      uint32_t th_emit, uint32_t th_tie, int tie_mode, bool hist_smem,
                      bool hist) -> mad_status {
    SpRowParams p{};
    p.aptr = A->rowptr;
    p.acol = A->colidx;
    p.rows = w.rorder;
    p.nrows_bins = bins;
    p.nrows_cap = rows_cap;
    p.bptr = w.bp;
    p.bcol = w.bcol;
    p.nlab = nlab;
    p.sel = w.sel;
    p.pre = w.pre;
    p.colmap = w.colmap;
    p.gram = gram;
    p.excl = excl;
    p.window = nlab < kSpWindowMax ? ((nlab + 31) & ~31u) : kSpWindowMax;
    if (p.window == 0) p.window = 32;
    p.th_emit = th_emit;
    p.th_tie = th_tie;
    p.tie_mode = tie_mode;
    p.tiecnt = w.tiecnt;
    p.hist_smem = hist_smem;
    p.hist = hist ? w.hist : nullptr;
    p.hist_bins = hist_smem ? kHistSmem : kHistGlobal;
    p.list = w.sel_ws.l0;
    p.cap = kSpListCap;
    p.sc = w.sc;
    const size_t smem = (size_t)p.window * 4 + (hist_smem ? (size_t)kHistSmem * 4 : 0);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spgemm_rowblock_topk, kSpBlock, smem);
    if (per_sm < 1) per_sm = 1;
    uint64_t blocks = (uint64_t)per_sm * sms;
    if (blocks > rows_cap) blocks = rows_cap ? rows_cap : 1;
    cudaMemsetAsync(&w.sc->row_next, 0, sizeof(unsigned int), st);
    k_spgemm_rowblock_topk<<<(unsigned)blocks, kSpBlock, smem, st>>>(p);
    count_launch(ctx);
    return cuda_status(cudaGetLastError());
  };

  // 1. Pilot: the heaviest rows against the heaviest columns, every stored
  //    entry counted into the histogram; its t-th largest is theta_0.
  const uint32_t hr = (uint32_t)(rows_nz < kPilot ? rows_nz : kPilot);
  const uint32_t hc = (uint32_t)(cols_nz < kPilot ? cols_nz : kPilot);
  if ((rs = select_columns(true, hc, 0)) != MAD_OK) return rs;
  cudaMemsetAsync(w.hist, 0, 4 * kHistGlobal, st);
  // The pilot's rows are the first hr of the row order: count them through
  // a bucket array that sums to hr.
  unsigned int* pilot_bins = w.hist + kHistGlobal - 32;
  {
    unsigned int hb[32] = {0};
    hb[0] = hr;
    cudaMemcpyAsync(pilot_bins, hb, sizeof(hb), cudaMemcpyHostToDevice, st);
  }
  if ((rs = run_rows(hc, pilot_bins, hr, 1u, 0u, 0, true, true)) != MAD_OK) return rs;
  k_hist_theta<<<1, 1024, 0, st>>>(w.hist, kHistSmem, t, w.sc);
  count_launch(ctx);
  unsigned int theta0 = 1;
  cudaMemcpyAsync(&theta0, &w.sc->theta, 4, cudaMemcpyDeviceToHost, st);
  if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(ce);

  // 2. Main pass over the rows and columns that can reach theta_0.
  const uint32_t th_deg = bound ? theta0 : 1u;
  cudaMemsetAsync(w.sc, 0, sizeof(SpScalars), st);
  k_logbin_count<<<blocks_for(m, grid_stream), 256, 0, st>>>(A->rowptr, nullptr, m, th_deg,
                                                            w.sc->bins[0]);
  k_logbin_scatter<<<blocks_for(m, grid_stream), 256, 0, st>>>(A->rowptr, nullptr, m, th_deg,
                                                              w.sc->bins[0], w.sc->cur[0],
                                                              w.rorder);
  count_launch(ctx, 2);
  if ((rs = select_columns(false, 0, th_deg)) != MAD_OK) return rs;
  uint32_t nlab = 0;
  cudaMemcpyAsync(&nlab, w.pre + n, 4, cudaMemcpyDeviceToHost, st);
  cudaMemsetAsync(w.hist, 0, 4 * kHistGlobal, st);
  if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(ce);
  if (nlab > 0) {
    if ((rs = run_rows(nlab, w.sc->bins[0], (uint32_t)m, theta0, 0u, 0, false, true)) != MAD_OK)
      return rs;
  }
  unsigned long long count = 0;
  cudaMemcpyAsync(&count, &w.sc->count, 8, cudaMemcpyDeviceToHost, st);
  if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(ce);

  if (count > kSpListCap) {
    // Too many candidates at theta_0: the exact tau from the histogram,
    // then every c > tau and the smallest keys among c == tau.
    k_hist_theta<<<1, 1024, 0, st>>>(w.hist, kHistGlobal, t, w.sc);
    count_launch(ctx);
    unsigned int tau = 0;
    cudaMemcpyAsync(&tau, &w.sc->theta, 4, cudaMemcpyDeviceToHost, st);
    if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(ce);
    if (tau >= kHistGlobal - 1) return MAD_ERR_UNSUPPORTED;   // counts beyond the histogram
    cudaMemsetAsync(&w.sc->count, 0, 8, st);
    cudaMemsetAsync(w.tiecnt, 0, 8 * (m + 1), st);
    if ((rs = run_rows(nlab, w.sc->bins[0], (uint32_t)m, tau + 1, tau, 1, false, false)) != MAD_OK)
      return rs;
    if ((rs = scan_exclusive_u64(ctx, (const uint64_t*)w.tiecnt, (uint64_t*)w.tiepre, m, (uint64_t*)w.part64, st)) != MAD_OK) return rs;
    k_tie_limit<<<blocks_for(m, grid_stream), 256, 0, st>>>(w.tiepre, m, t, w.sc);
    count_launch(ctx);
    if ((rs = run_rows(nlab, w.sc->bins[0], (uint32_t)m, 0xffffffffu, tau, 2, false, false)) !=
        MAD_OK)
      return rs;
    cudaMemcpyAsync(&count, &w.sc->count, 8, cudaMemcpyDeviceToHost, st);
    if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(ce);
    if (count > kSpListCap) return MAD_ERR_STATE;
  }

  // 3. The t largest candidates by (c desc, key asc).
  uint64_t nsel = 0;
  if ((rs = select_list(ctx, w.sel_ws, count, t, 4, &nsel, st)) != MAD_OK) return rs;
  if (nsel) {
    k_sp_to_pairs<<<blocks_for(nsel, 1u << 30), 256, 0, st>>>(w.sel_ws.out, nsel, out_dev);
    count_launch(ctx);
  }
  if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(ce);
  *n_out_host = (uint32_t)nsel;
  return MAD_OK;
}
