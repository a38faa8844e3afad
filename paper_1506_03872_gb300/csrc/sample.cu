// The sampling loop of Alg. 2: for every diamond index l, draw the center
// edge (i,k) with probability w_ik / ||W||_1 (two stages: row i from T1,
// then k from row i of T2), j with probability |b_kj| / ||b_k*||_1 (row k of
// TB), k' with probability |a_ik'| / ||a_i*||_1 (row i of TA), and add
// sgn(a_ik b_kj a_ik') b_k'j to x_ij (Alg. 2 increment line).
//
// GPU organisation: one diamond per thread, grid-stride over the diamond
// range with a warp-uniform trip count; the signs of a_ik, b_kj and a_ik'
// come for free with the table entries the searches land on (bit 31), so
// only b_k'j is read from B.  Lanes of a warp whose diamonds hit the same
// key combine their increments before one lane inserts into the hash.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "mad_device.cuh"
#include "mad_internal.cuh"

namespace mad {
namespace {

struct Draw {
  uint32_t i, k, j, kp;
  long long v;
};

__device__ __forceinline__ Draw draw_one(const SampleParams& p, unsigned long long seed,
                                         unsigned long long ell, bool* bad) {
  const Uniforms u = diamond_uniforms(seed, ell);
  const uint32_t mask = p.integer ? 0xFFFFFFFFu : PREFIX_MASK;
  // Center edge, stage 1: row i of A.
  const int64_t i = search_u64(p.T1, p.m, draw_target(u.u0, p.t1_total), bad);
  int64_t a0, alen;
  if (p.dense) {
    a0 = i * p.d;
    alen = p.d;
  } else {
    a0 = __ldg(p.a_ptr + i);
    alen = __ldg(p.a_ptr + i + 1) - a0;
  }
  // Center edge, stage 2: k within row i.
  const uint32_t t2tot = __ldg(p.T2 + a0 + alen - 1) & mask;
  const int64_t pk = search_u32(p.T2 + a0, alen, (uint32_t)draw_target(u.u1, t2tot), mask, bad);
  const uint32_t e_k = __ldg(p.T2 + a0 + pk);
  const int64_t k = p.dense ? pk : (int64_t)__ldg(p.a_col + a0 + pk);
  // j from row k of B.
  int64_t b0, blen;
  if (p.dense) {
    b0 = k * p.n;
    blen = p.n;
  } else {
    b0 = __ldg(p.b_ptr + k);
    blen = __ldg(p.b_ptr + k + 1) - b0;
  }
  int64_t pj;
  uint32_t e_j = 0;
  if (p.integer) {
    pj = (int64_t)draw_target(u.u2, (unsigned long long)blen);
  } else {
    const uint32_t tbtot = __ldg(p.TB + b0 + blen - 1) & mask;
    pj = search_u32(p.TB + b0, blen, (uint32_t)draw_target(u.u2, tbtot), mask, bad);
    e_j = __ldg(p.TB + b0 + pj);
  }
  const int64_t j = p.dense ? pj : (int64_t)__ldg(p.b_col + b0 + pj);
  // k' from row i of A.
  int64_t pkp;
  uint32_t e_kp = 0;
  if (p.integer) {
    pkp = (int64_t)draw_target(u.u3, (unsigned long long)alen);
  } else {
    const uint32_t tatot = __ldg(p.TA + a0 + alen - 1) & mask;
    pkp = search_u32(p.TA + a0, alen, (uint32_t)draw_target(u.u3, tatot), mask, bad);
    e_kp = __ldg(p.TA + a0 + pkp);
  }
  const int64_t kp = p.dense ? pkp : (int64_t)__ldg(p.a_col + a0 + pkp);
  // Increment.
  long long v;
  if (p.integer) {
    const int64_t c0 = __ldg(p.b_ptr + kp), clen = __ldg(p.b_ptr + kp + 1) - c0;
    bool hit;
    if (p.flags & MAD_GRAM) {
      // B = A^T: b_k'j = a_jk'; search the shorter of the two sorted rows.
      const int64_t r0 = __ldg(p.a_ptr + j), rlen = __ldg(p.a_ptr + j + 1) - r0;
      hit = (rlen < clen) ? contains_sorted(p.a_col + r0, rlen, (int32_t)kp)
                          : contains_sorted(p.b_col + c0, clen, (int32_t)j);
    } else {
      hit = contains_sorted(p.b_col + c0, clen, (int32_t)j);
    }
    v = hit ? 1 : 0;
  } else {
    const int64_t off = kp * p.ldb + j;
    const float b = p.b_f64 ? __double2float_rn(__ldg((const double*)p.b_val + off))
                            : __ldg((const float*)p.b_val + off);
    v = __double2ll_rn((double)b * p.f_scale);
    if (!(p.flags & MAD_NONNEG) && ((e_k ^ e_j ^ e_kp) & SIGN_BIT)) v = -v;
  }
  Draw dr;
  dr.i = (uint32_t)i;
  dr.k = (uint32_t)k;
  dr.j = (uint32_t)j;
  dr.kp = (uint32_t)kp;
  dr.v = v;
  return dr;
}

__global__ void __launch_bounds__(256)
k_sample(const SampleParams p, unsigned long long seed, unsigned long long first,
         unsigned long long s) {
  const int lane = threadIdx.x & 31;
  const unsigned long long warp_id = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long inserted = 0, diag = 0, created = 0;
  bool bad = false, full = false;
  for (unsigned long long base = warp_id * 32; base < s; base += warps * 32) {
    const unsigned long long q = base + lane;
    bool want = false;
    unsigned long long key = 0;
    long long v = 0;
    if (q < s) {
      const Draw dr = draw_one(p, seed, first + q, &bad);
      if ((p.flags & MAD_EXCLUDE_DIAG) && dr.i == dr.j) {
        ++diag;
      } else if (dr.v != 0) {
        uint32_t a = dr.i, b = dr.j;
        if ((p.flags & MAD_GRAM) && b < a) {
          a = dr.j;
          b = dr.i;
        }
        key = ((unsigned long long)a << 32) | b;
        v = dr.v;
        want = true;
        ++inserted;
      }
    }
    const unsigned active = __ballot_sync(0xFFFFFFFFu, want);
    if (want) {
      const unsigned peers = __match_any_sync(active, key);
      long long total = 0;
      unsigned rem = peers;
      while (rem) {
        const int src = __ffs(rem) - 1;
        total += __shfl_sync(peers, v, src);
        rem &= rem - 1;
      }
      if (lane == __ffs(peers) - 1) {
        const int r = hash_add(p.hkeys, p.hvals, p.hmask, p.max_probe, key, total);
        if (r == 0) full = true;
        if (r == 2) ++created;
      }
    }
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    inserted += __shfl_xor_sync(0xFFFFFFFFu, inserted, off);
    diag += __shfl_xor_sync(0xFFFFFFFFu, diag, off);
    created += __shfl_xor_sync(0xFFFFFFFFu, created, off);
  }
  const unsigned any_bad = __ballot_sync(0xFFFFFFFFu, bad);
  const unsigned any_full = __ballot_sync(0xFFFFFFFFu, full);
  if (lane == 0) {
    if (inserted) atomicAdd(&p.sc->inserted, inserted);
    if (diag) atomicAdd(&p.sc->diag_skipped, diag);
    if (created) atomicAdd(&p.sc->new_keys, created);
    if (any_bad) atomicOr(&p.sc->err, DERR_SEARCH);
    if (any_full) atomicOr(&p.sc->err, DERR_HASH_FULL);
  }
}

// Diagnostic twin of k_sample: writes each diamond's draws instead of
// accumulating them.
__global__ void __launch_bounds__(256)
k_draws(const SampleParams p, unsigned long long seed, unsigned long long first,
        const unsigned long long* __restrict__ ells, unsigned long long count, uint32_t* oi,
        uint32_t* ok, uint32_t* oj, uint32_t* okp, long long* ov) {
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

int sample_grid(unsigned long long s) {
  static int blocks_per_sm = -1, sms = 0;
  if (blocks_per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_sample, 256, 0) !=
            cudaSuccess ||
        blocks_per_sm < 1)
      blocks_per_sm = 1;
  }
  const unsigned long long need = (s + 255) / 256;
  const unsigned long long full = (unsigned long long)sms * blocks_per_sm;
  return (int)(need < full ? (need ? need : 1) : full);
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
  p.f_scale = std::ldexp(1.0, ctx->f);
  p.hkeys = ctx->hkeys;
  p.hvals = ctx->hvals;
  p.hmask = ctx->hcap - 1;
  p.max_probe = (uint32_t)(ctx->hcap < 4096 ? ctx->hcap : 4096);
  p.dense = ctx->dense ? 1 : 0;
  p.a_f64 = ctx->A.dt == MAD_F64;
  p.b_f64 = ctx->B.dt == MAD_F64;
  p.integer = ctx->integer ? 1 : 0;
  p.flags = ctx->flags;
  p.sc = ctx->sc;
  return p;
}

mad_status sample_impl(mad_ctx* ctx, uint64_t s, uint64_t seed, uint64_t first, cudaStream_t st) {
  if (s == 0) return MAD_OK;
  const SampleParams p = make_params(ctx);
  k_sample<<<sample_grid(s), 256, 0, st>>>(p, seed, first, s);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

mad_status debug_draws_impl(mad_ctx* ctx, uint64_t seed, uint64_t first, const uint64_t* ells,
                            uint64_t count, uint32_t* oi, uint32_t* ok, uint32_t* oj,
                            uint32_t* okp, int64_t* ov, cudaStream_t st) {
  if (count == 0) return MAD_OK;
  const SampleParams p = make_params(ctx);
  const unsigned long long blocks = (count + 255) / 256;
  k_draws<<<(unsigned)(blocks < 152 * 8 ? blocks : 152 * 8), 256, 0, st>>>(
      p, seed, first, (const unsigned long long*)ells, count, oi, ok, oj, okp, (long long*)ov);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

}  // namespace mad
