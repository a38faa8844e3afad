// Batched queries: many instances A = Q[q] (1 x d) against one item matrix B
// (d x n), each a complete run of Alg. 2 and Alg. 3 with its own budget.
//
// With m = 1 the stage-1 draw of the center edge always returns the query's
// row, so diamond l of query q needs only the uniforms of k, j and k' (the
// Philox stream of seed + q, counter l, exactly as a single-query run) and
// the rest of the loop body is the dense path's: k from the query's T2 row,
// j from row k of TB (a guided search: n is large), k' from its TA row, the
// increment from B.  Diamonds come in 256-diamond chunks that never mix
// queries, so a warp's diamonds share the query's T2/TA rows and its hash
// region; each query's keys stay inside its region (probing wraps there),
// so Alg. 3 runs per query on the region alone: one CTA selects the t'
// largest positive x, rescores them exactly and keeps the t largest |c|.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "draw.cuh"
#include "mad_device.cuh"
#include "mad_internal.cuh"

namespace mad {
namespace {

constexpr int kChunk = 256;       // diamonds per chunk (one per thread)
constexpr int kSelCap = 4096;     // candidates a query's selection keeps
constexpr int kTPrimeMax = 1024;  // largest t' of a batch

// Hash insert into query q's region [hreg[q], hreg[q+1]) (a power of two of
// at least 4 slots, 4-aligned), probing inside the region only.
__device__ __forceinline__ int region_add(const SampleParams& p, uint32_t q,
                                          unsigned long long key, long long v) {
  const unsigned long long r0 = __ldg(p.hreg + q), r1 = __ldg(p.hreg + q + 1);
  const unsigned long long size = r1 - r0;
  const uint64_t home = r0 + (mix64(key) & (size - 1));
  return hash_add_from(p.hkeys, p.hvals, r0, r1, home, (uint32_t)size, key, v);
}

// Alg. 2 over every query's diamonds: chunk c holds diamonds l0 .. l0+255 of
// query chunk_q[c] (the last chunk of a query is partial).
__global__ void __launch_bounds__(256, 4)
k_mips_sample(const SampleParams p, unsigned long long seed, const uint32_t* __restrict__ chunk_q,
              const uint32_t* __restrict__ chunk_l0, const unsigned long long* __restrict__ s_q,
              unsigned long long nchunks, int mult) {
  bool bad = false, full = false;
  unsigned long long inserted = 0, created = 0;
  for (unsigned long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const uint32_t q = __ldg(chunk_q + c);
    const unsigned long long sq = __ldg(s_q + q);
    for (int rep = 0; rep < mult; ++rep) {
      const unsigned long long l =
          (unsigned long long)__ldg(chunk_l0 + c) + threadIdx.x + (unsigned long long)rep * kChunk;
      if (l >= sq) break;
      const Uniforms u = diamond_uniforms(seed + q, l);
      const Draw dr = draw_given_row(p, u, (int64_t)q, &bad);
      if (dr.v != 0) {
        ++inserted;
        const int r = region_add(p, q, ((unsigned long long)q << 32) | dr.j, dr.v);
        if (r == 0) full = true;
        if (r == 2) ++created;
      }
    }
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    inserted += __shfl_xor_sync(0xFFFFFFFFu, inserted, off);
    created += __shfl_xor_sync(0xFFFFFFFFu, created, off);
  }
  const unsigned any_bad = __ballot_sync(0xFFFFFFFFu, bad);
  const unsigned any_full = __ballot_sync(0xFFFFFFFFu, full);
  if ((threadIdx.x & 31) == 0) {
    if (inserted) atomicAdd(&p.sc->inserted, inserted);
    if (created) atomicAdd(&p.sc->new_keys, created);
    if (any_bad) atomicOr(&p.sc->err, DERR_SEARCH);
    if (any_full) atomicOr(&p.sc->err, DERR_HASH_FULL);
  }
}

// Bitonic sort of n (a power of two, <= kSelCap) entries of shared arrays
// into "before" order; all threads of the block take part.
template <typename Before>
__device__ void block_bitonic(unsigned long long* a, unsigned long long* b, double* c, int n,
                              Before before) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
        const int x = ((t & ~(j - 1)) << 1) | (t & (j - 1)), y = x + j;   // j a power of two
        const bool up = (x & k) == 0;
        const bool y_first = before(a[y], b[y], c ? c[y] : 0.0, a[x], b[x], c ? c[x] : 0.0);
        if (y_first == up) {
          const unsigned long long ta = a[x], tb = b[x];
          a[x] = a[y]; b[x] = b[y]; a[y] = ta; b[y] = tb;
          if (c) {
            const double tc = c[x];
            c[x] = c[y];
            c[y] = tc;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Offset of v inside its log bucket, scaled to 10 bits (monotone in v).
__device__ __forceinline__ uint32_t fine_of(unsigned long long v, uint32_t b) {
  const int e = 63 - __clzll((long long)v);
  const int sh = e > 14 ? e - 14 : 0;
  const unsigned long long f = (v - bucket_floor(b)) >> sh;
  return f < 1024 ? (uint32_t)f : 1023u;
}

// Alg. 3 for query blockIdx.x over its hash region.  The t' largest positive
// x by (x desc, key asc): a log-bucket histogram finds the bucket where the
// count from the top reaches t', a 10-bit histogram inside that bucket
// narrows it, and every x at or above the resulting threshold (all of the
// top t', and few more) is collected and sorted.  Then c = q . b_j in FP64
// (32 lane-strided fused multiply-add partial sums folded in halves) and the
// t largest |c| by (|c| desc, key asc).
__global__ void __launch_bounds__(512)
k_mips_select(const unsigned long long* __restrict__ hkeys, const long long* __restrict__ hvals,
              const unsigned long long* __restrict__ hreg, const float* __restrict__ Q,
              int64_t ldq, const float* __restrict__ Bt, int64_t d, uint32_t tprime, uint32_t t,
              mad_pair* __restrict__ out, uint32_t* __restrict__ nout,
              mad_pair* __restrict__ cand_out, DevScalars* sc) {
  extern __shared__ unsigned long long sel_smem[];
  unsigned long long* cx = sel_smem;            // x of the collected keys
  unsigned long long* ck = sel_smem + kSelCap;  // keys
  double* cc = (double*)(sel_smem + 2 * kSelCap);  // c of the top t'
  __shared__ unsigned int hist[1024];
  __shared__ unsigned int fine[1024];
  __shared__ int bstar, fstar;
  __shared__ unsigned int ncol;
  __shared__ unsigned long long above;
  const uint32_t q = blockIdx.x;
  const unsigned long long r0 = hreg[q], r1 = hreg[q + 1];
  for (int b = threadIdx.x; b < 1024; b += blockDim.x) hist[b] = fine[b] = 0;
  if (threadIdx.x == 0) {
    ncol = 0;
    above = 0;
  }
  __syncthreads();
  for (unsigned long long s = r0 + threadIdx.x; s < r1; s += blockDim.x) {
    const long long v = hvals[s];
    if (v > 0) atomicAdd(&hist[log_bucket((unsigned long long)v)], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long cum = 0;
    int pick = -1;
    for (int b = 1023; b >= 0; --b) {
      if (cum + hist[b] >= tprime) {
        pick = b;
        break;
      }
      cum += hist[b];
    }
    bstar = pick;
    above = cum;
  }
  __syncthreads();
  const int bs = bstar;
  if (bs >= 0) {
    for (unsigned long long s = r0 + threadIdx.x; s < r1; s += blockDim.x) {
      const long long v = hvals[s];
      if (v > 0 && log_bucket((unsigned long long)v) == (uint32_t)bs)
        atomicAdd(&fine[fine_of((unsigned long long)v, (uint32_t)bs)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long cum = above;
      int pick = 0;
      for (int f = 1023; f >= 0; --f) {
        cum += fine[f];
        if (cum >= tprime) {
          pick = f;
          break;
        }
      }
      fstar = pick;
    }
    __syncthreads();
  }
  const int fs = bs >= 0 ? fstar : 0;
  for (unsigned long long s = r0 + threadIdx.x; s < r1; s += blockDim.x) {
    const long long v = hvals[s];
    if (v <= 0) continue;
    bool take = true;
    if (bs >= 0) {
      const uint32_t b = log_bucket((unsigned long long)v);
      take = b > (uint32_t)bs || (b == (uint32_t)bs && fine_of((unsigned long long)v, b) >= (uint32_t)fs);
    }
    if (take) {
      const unsigned pos = atomicAdd(&ncol, 1u);
      if (pos < kSelCap) {
        cx[pos] = (unsigned long long)v;
        ck[pos] = hkeys[s];
      }
    }
  }
  __syncthreads();
  const unsigned n_all = ncol;
  if (n_all > kSelCap && threadIdx.x == 0) atomicOr(&sc->err, DERR_SELECT);
  const int n = (int)(n_all < kSelCap ? n_all : kSelCap);
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int x = n + threadIdx.x; x < n2; x += blockDim.x) {
    cx[x] = 0;           // sorts after every collected x (all positive)
    ck[x] = ~0ull;
  }
  __syncthreads();
  block_bitonic(cx, ck, (double*)nullptr, n2,
                [](unsigned long long ax, unsigned long long ak, double, unsigned long long bx,
                   unsigned long long bk, double) { return ax > bx || (ax == bx && ak < bk); });
  const int K = n < (int)tprime ? n : (int)tprime;
  if (cand_out) {
    for (int x = threadIdx.x; x < K; x += blockDim.x) {
      mad_pair pr;
      pr.i = q;
      pr.j = (uint32_t)ck[x];
      pr.x = (int64_t)cx[x];
      pr.c = 0.0;
      cand_out[(size_t)q * tprime + x] = pr;
    }
  }
  // Exact rescoring, one warp per candidate.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  const float* __restrict__ a = Q + (int64_t)q * ldq;
  for (int x = warp; x < K; x += warps) {
    const float* __restrict__ b = Bt + (int64_t)(uint32_t)ck[x] * d;
    double acc = 0.0;
    for (int64_t k = lane; k < d; k += 32) acc = __fma_rn((double)a[k], (double)b[k], acc);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, off));
    if (lane == 0) cc[x] = acc;
  }
  __syncthreads();
  // The t largest |c| among the K: sort the K by (|c| desc, key asc).
  int k2 = 1;
  while (k2 < K) k2 <<= 1;
  for (int x = K + threadIdx.x; x < k2; x += blockDim.x) {
    cx[x] = 0;
    ck[x] = ~0ull;
    cc[x] = -1.0;   // |c| of a padding entry is below every real |c|
  }
  __syncthreads();
  if (K > 1)
    block_bitonic(cx, ck, cc, k2,
                  [](unsigned long long, unsigned long long ak, double ac, unsigned long long,
                     unsigned long long bk, double bc) {
                    const double fa = ac < 0.0 && ak == ~0ull ? -1.0 : fabs(ac);
                    const double fb = bc < 0.0 && bk == ~0ull ? -1.0 : fabs(bc);
                    return fa > fb || (fa == fb && ak < bk);
                  });
  const int T = K < (int)t ? K : (int)t;
  for (int x = threadIdx.x; x < T; x += blockDim.x) {
    mad_pair pr;
    pr.i = q;
    pr.j = (uint32_t)ck[x];
    pr.x = (int64_t)cx[x];
    pr.c = cc[x];
    out[(size_t)q * t + x] = pr;
  }
  if (threadIdx.x == 0) nout[q] = (uint32_t)T;
}

// Region of query q: a power of two >= max(4, 2^lg s_q) slots.
__global__ void __launch_bounds__(256)
k_mips_region_sizes(const unsigned long long* __restrict__ s_q, uint32_t nq, int lg,
                    unsigned long long* __restrict__ sizes) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    unsigned long long size = 4;
    while (size < (s_q[q] << lg)) size <<= 1;
    sizes[q] = size;
  }
}

template <typename T>
mad_status pool_alloc(mad_ctx* ctx, T*& p, size_t count, cudaStream_t st) {
  if (count == 0) count = 1;
  void* q = nullptr;
  const mad_status rs = pool_malloc(ctx, &q, count * sizeof(T), st);
  p = (T*)q;
  return rs;
}

template <typename T>
void pool_free(T*& p, cudaStream_t st) {
  if (p) cudaFreeAsync((void*)p, st);
  p = nullptr;
}

size_t select_smem_bytes() { return (size_t)kSelCap * 16 + (size_t)kTPrimeMax * 8; }

}  // namespace
}  // namespace mad

using namespace mad;

extern "C" {

mad_status mad_mips_items(mad_ctx* ctx, const mad_matrix* B, uint64_t s_max, mad_stream stream) {
  if (!ctx || !B || s_max == 0 || s_max > (1ull << 40)) return MAD_ERR_ARG;
  if (B->fmt != MAD_DENSE_ROWMAJOR || B->dt != MAD_F32 || !B->values || B->rows <= 0 ||
      B->cols <= 0 || B->ld < B->cols)
    return MAD_ERR_ARG;
  if (B->cols >= (1ll << 31) || B->rows > 1024) return MAD_ERR_UNSUPPORTED;
  if (ctx->flags) return MAD_ERR_UNSUPPORTED;   // plain |q . b_j|, no Gram or sign flags
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamSynchronize(st);
  // Drop every earlier table (single-instance or batched).
  pool_free(ctx->T1, st); pool_free(ctx->T2, st); pool_free(ctx->TA, st); pool_free(ctx->TB, st);
  pool_free(ctx->na, st); pool_free(ctx->nb, st); pool_free(ctx->r, st); pool_free(ctx->r64, st);
  pool_free(ctx->bt, st); pool_free(ctx->hkeys, st); pool_free(ctx->hvals, st);
  pool_free(ctx->hreg, st); pool_free(ctx->T2g_ptr, st);
  pool_free(ctx->T2g, st); pool_free(ctx->T2g_sh, st); pool_free(ctx->bloom, st);
  pool_free(ctx->TBg, st); pool_free(ctx->TBg_sh, st);
  pool_free(ctx->mips_s, st); pool_free(ctx->mips_chunk_q, st); pool_free(ctx->mips_chunk_l0, st);
  pool_free(ctx->pipe_buf, st);
  pool_free(ctx->pipe_scratch, st);
  ctx->pipe_scratch_bytes = 0;
  ctx->pipe = false;
  ctx->built = false;
  ctx->mips_items = false;
  ctx->mips_nq = 0;
  ctx->B = *B;
  ctx->dense = true;
  ctx->integer = false;
  ctx->regioned = true;
  ctx->hov = 0;
  ctx->d = B->rows;
  ctx->n = B->cols;
  ctx->m = 0;
  ctx->s_max = s_max;
  mad_status rs;
  if ((rs = pool_alloc(ctx, ctx->TB, (size_t)(ctx->d * ctx->n), st)) != MAD_OK) return rs;
  if ((rs = pool_alloc(ctx, ctx->nb, (size_t)ctx->d, st)) != MAD_OK) return rs;
  char* bt = nullptr;
  if ((rs = pool_alloc(ctx, bt, (size_t)(ctx->n * ctx->d) * 4, st)) != MAD_OK) return rs;
  ctx->bt = bt;
  ctx->tbg_stride = ((int64_t)1 << tb_guide_width(ctx->n)) + 1;
  if ((rs = pool_alloc(ctx, ctx->TBg_sh, (size_t)ctx->d, st)) != MAD_OK) return rs;
  if ((rs = pool_alloc(ctx, ctx->TBg, (size_t)(ctx->d * ctx->tbg_stride), st)) != MAD_OK) return rs;
  cudaMemsetAsync(ctx->sc, 0, sizeof(DevScalars), st);
  if ((rs = build_item_tables(ctx, st)) != MAD_OK) return rs;
  if ((rs = tb_guide_build(ctx, st)) != MAD_OK) return rs;
  DevScalars hs;
  cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, st);
  if ((rs = cuda_status(cudaStreamSynchronize(st))) != MAD_OK) return rs;
  if (hs.maxb_bits == 0u) return MAD_ERR_EMPTY;
  float maxb;
  std::memcpy(&maxb, &hs.maxb_bits, sizeof(float));
  int lgs = 0;
  while (lgs < 64 && (1ull << lgs) < s_max) ++lgs;
  ctx->f = 62 - lgs - (std::ilogb(maxb) + 1);
  ctx->mips_items = true;
  return cuda_status(cudaStreamSynchronize(st));
}

mad_status mad_mips_config(mad_ctx* ctx, uint32_t region_lg, uint32_t chunk_mult,
                           uint32_t blocks_per_sm, uint32_t select_threads) {
  if (!ctx || region_lg > 4 || blocks_per_sm > 8) return MAD_ERR_ARG;
  if (chunk_mult != 0 && chunk_mult != 1 && chunk_mult != 2 && chunk_mult != 4 && chunk_mult != 8)
    return MAD_ERR_ARG;
  if (select_threads != 0 && select_threads != 128 && select_threads != 256 &&
      select_threads != 512)
    return MAD_ERR_ARG;
  ctx->mips_region_lg = region_lg == 0 ? 1 : (int)region_lg;
  ctx->mips_chunk_mult = chunk_mult == 0 ? 1 : (int)chunk_mult;
  ctx->mips_bps = (int)blocks_per_sm;
  ctx->mips_select_threads = select_threads == 0 ? 256 : (int)select_threads;
  return MAD_OK;
}

mad_status mad_mips_plan(mad_ctx* ctx, uint32_t nq, const uint64_t* s_host, uint32_t tprime,
                         uint32_t t, mad_stream stream) {
  if (!ctx || !s_host || nq == 0 || tprime == 0 || tprime > (uint32_t)kTPrimeMax || t == 0 ||
      t > tprime)
    return MAD_ERR_ARG;
  if (!ctx->mips_items) return MAD_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint32_t> cq, cl;
  uint64_t chunks = 0;
  const uint64_t csize = (uint64_t)kChunk * (uint64_t)ctx->mips_chunk_mult;
  for (uint32_t q = 0; q < nq; ++q) {
    if (s_host[q] == 0 || s_host[q] > ctx->s_max) return MAD_ERR_ARG;
    chunks += (s_host[q] + csize - 1) / csize;
  }
  cq.reserve(chunks);
  cl.reserve(chunks);
  for (uint32_t q = 0; q < nq; ++q)
    for (uint64_t l = 0; l < s_host[q]; l += csize) {
      cq.push_back(q);
      cl.push_back((uint32_t)l);
    }
  cudaStreamSynchronize(st);
  pool_free(ctx->T2, st); pool_free(ctx->TA, st); pool_free(ctx->na, st); pool_free(ctx->r, st);
  pool_free(ctx->hkeys, st); pool_free(ctx->hvals, st); pool_free(ctx->hreg, st);
  pool_free(ctx->mips_s, st); pool_free(ctx->mips_chunk_q, st); pool_free(ctx->mips_chunk_l0, st);
  ctx->mips_nq = 0;
  mad_status rs;
  if ((rs = pool_alloc(ctx, ctx->T2, (size_t)nq * (size_t)ctx->d, st)) != MAD_OK) return rs;
  if ((rs = pool_alloc(ctx, ctx->TA, (size_t)nq * (size_t)ctx->d, st)) != MAD_OK) return rs;
  if ((rs = pool_alloc(ctx, ctx->na, (size_t)nq, st)) != MAD_OK) return rs;
  if ((rs = pool_alloc(ctx, ctx->r, (size_t)nq, st)) != MAD_OK) return rs;
  if ((rs = pool_alloc(ctx, ctx->hreg, (size_t)nq + 1, st)) != MAD_OK) return rs;
  if ((rs = pool_alloc(ctx, ctx->mips_s, (size_t)nq, st)) != MAD_OK) return rs;
  if ((rs = pool_alloc(ctx, ctx->mips_chunk_q, (size_t)chunks, st)) != MAD_OK) return rs;
  if ((rs = pool_alloc(ctx, ctx->mips_chunk_l0, (size_t)chunks, st)) != MAD_OK) return rs;
  cudaMemcpyAsync(ctx->mips_s, s_host, nq * sizeof(uint64_t), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(ctx->mips_chunk_q, cq.data(), chunks * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(ctx->mips_chunk_l0, cl.data(), chunks * sizeof(uint32_t), cudaMemcpyHostToDevice,
                  st);
  // Regions: sizes, then their offsets (hreg[nq] = total).
  const size_t sizes_bytes = ((size_t)nq * 8 + 255) & ~(size_t)255;
  if ((rs = ensure_scratch(ctx, sizes_bytes + scan_partial_elems(nq) * 8, st)) != MAD_OK) return rs;
  unsigned long long* sizes = (unsigned long long*)ctx->scratch;
  uint64_t* part = (uint64_t*)((char*)ctx->scratch + sizes_bytes);
  k_mips_region_sizes<<<(nq + 255) / 256, 256, 0, st>>>(ctx->mips_s, nq, ctx->mips_region_lg,
                                                       sizes);
  count_launch(ctx);
  if ((rs = scan_exclusive_u64(ctx, (const uint64_t*)sizes, (uint64_t*)ctx->hreg, nq, part, st)) !=
      MAD_OK)
    return rs;
  unsigned long long total = 0;
  cudaMemcpyAsync(&total, ctx->hreg + nq, sizeof(total), cudaMemcpyDeviceToHost, st);
  if ((rs = cuda_status(cudaStreamSynchronize(st))) != MAD_OK) return rs;
  if ((rs = pool_alloc(ctx, ctx->hkeys, (size_t)total, st)) != MAD_OK) return rs;
  if ((rs = pool_alloc(ctx, ctx->hvals, (size_t)total, st)) != MAD_OK) return rs;
  ctx->hcap = ctx->hcap_alloc = total;
  ctx->m = nq;
  ctx->mips_nq = nq;
  ctx->mips_tprime = tprime;
  ctx->mips_t = t;
  ctx->mips_chunks = chunks;
  ctx->mips_plan_mult = ctx->mips_chunk_mult;
  if (cudaFuncSetAttribute(k_mips_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)select_smem_bytes()) != cudaSuccess)
    return MAD_ERR_CUDA;
  return cuda_status(cudaStreamSynchronize(st));
}

mad_status mad_mips_run(mad_ctx* ctx, const mad_matrix* Q, uint64_t seed, mad_pair* out_dev,
                        uint32_t* n_out_dev, mad_pair* cand_dev, mad_stream stream) {
  if (!ctx || !Q || !out_dev || !n_out_dev) return MAD_ERR_ARG;
  if (!ctx->mips_items || ctx->mips_nq == 0) return MAD_ERR_STATE;
  if (Q->fmt != MAD_DENSE_ROWMAJOR || Q->dt != MAD_F32 || !Q->values ||
      Q->rows != (int64_t)ctx->mips_nq || Q->cols != ctx->d || Q->ld < Q->cols)
    return MAD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->A = *Q;
  // Query rows of the tables (T2, TA; T1 is not needed: m = 1 per query).
  mad_status rs;
  if ((rs = build_query_rows(ctx, st)) != MAD_OK) return rs;
  cudaMemsetAsync(ctx->hkeys, 0xFF, ctx->hcap * sizeof(unsigned long long), st);
  cudaMemsetAsync(ctx->hvals, 0, ctx->hcap * sizeof(long long), st);
  SampleParams p = make_params(ctx);
  p.regioned = 1;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mips_sample, 256, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (ctx->mips_bps > 0 && ctx->mips_bps < per_sm) per_sm = ctx->mips_bps;
  const unsigned long long grid =
      std::min<unsigned long long>(ctx->mips_chunks, (unsigned long long)sms * per_sm);
  k_mips_sample<<<(unsigned)grid, 256, 0, st>>>(p, seed, ctx->mips_chunk_q, ctx->mips_chunk_l0,
                                                ctx->mips_s, ctx->mips_chunks,
                                                ctx->mips_plan_mult);
  k_mips_select<<<ctx->mips_nq, ctx->mips_select_threads, select_smem_bytes(), st>>>(
      ctx->hkeys, ctx->hvals, ctx->hreg, (const float*)Q->values, Q->ld, (const float*)ctx->bt,
      ctx->d, ctx->mips_tprime, ctx->mips_t, out_dev, n_out_dev, cand_dev, ctx->sc);
  count_launch(ctx, 2);
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
