// One pass of the loop body of Alg. 2 for a single diamond, shared by the
// sampling kernels (single instance and batched queries).
#ifndef MAD_DRAW_CUH_
#define MAD_DRAW_CUH_

#include "mad_device.cuh"
#include "mad_internal.cuh"

namespace mad {

struct Draw {
  uint32_t i, k, j, kp;
  long long v;
};

// Center edge, stage 1: row i of A from T1 (through its guide when built).
__device__ __forceinline__ int64_t draw_row_i(const SampleParams& p, unsigned long long u0,
                                              bool* bad) {
  const unsigned long long target = draw_target(u0, p.t1_total);
  if (p.T1g) {
    const int64_t i = ub_guided_u64(p.T1, p.m, p.T1g, p.t1g_sh, target);
    if (i >= p.m) {
      *bad = true;
      return p.m - 1;
    }
    return i;
  }
  return search_u64(p.T1, p.m, target, bad);
}

// The rest of the loop body for a diamond whose row i is known.
__device__ __forceinline__ Draw draw_given_row(const SampleParams& p, const Uniforms& u,
                                               int64_t i, bool* bad) {
  const uint32_t mask = p.integer ? 0xFFFFFFFFu : PREFIX_MASK;
  int64_t a0, alen;
  if (p.dense) {
    a0 = i * p.d;
    alen = p.d;
  } else {
    a0 = __ldg(p.a_ptr + i);
    alen = __ldg(p.a_ptr + i + 1) - a0;
  }
  // Center edge, stage 2 (k within row i) and k' within row i: the two
  // searches run over rows of the same length, side by side.
  int64_t pk, pkp;
  uint32_t e_k, e_kp = 0;
  if (p.integer) {
    const uint32_t t2tot = __ldg(p.T2 + a0 + alen - 1);
    const uint32_t target = (uint32_t)draw_target(u.u1, t2tot);
    if (p.T2g && alen >= kGuideMin) {
      pk = ub_guided_u32(p.T2 + a0, p.T2g + __ldg(p.T2g_ptr + i), (int)__ldg(p.T2g_sh + i), target);
    } else {
      pk = ub_u32(p.T2 + a0, (int)alen, target, mask);
    }
    pkp = (int64_t)draw_target(u.u3, (unsigned long long)alen);
  } else {
    const uint32_t t2tot = __ldg(p.T2 + a0 + alen - 1) & mask;
    const uint32_t tatot = __ldg(p.TA + a0 + alen - 1) & mask;
    int a, b;
    ub2_u32(p.T2 + a0, p.TA + a0, (int)alen, (uint32_t)draw_target(u.u1, t2tot),
            (uint32_t)draw_target(u.u3, tatot), mask, &a, &b);
    pk = a;
    pkp = b;
  }
  if (pk >= alen) { *bad = true; pk = alen - 1; }
  if (pkp >= alen) { *bad = true; pkp = alen - 1; }
  e_k = __ldg(p.T2 + a0 + pk);
  if (!p.integer) e_kp = __ldg(p.TA + a0 + pkp);
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
    const uint32_t target = (uint32_t)draw_target(u.u2, tbtot);
    if (p.TBg) {
      pj = ub_guided_u32(p.TB + b0, p.TBg + k * p.tbg_stride, (int)__ldg(p.TBg_sh + k), target,
                         mask);
      if (pj >= blen) { *bad = true; pj = blen - 1; }
    } else {
      pj = ub_u32(p.TB + b0, (int)blen, target, mask);
      if (pj >= blen) { *bad = true; pj = blen - 1; }
    }
    e_j = __ldg(p.TB + b0 + pj);
  }
  const int64_t j = p.dense ? pj : (int64_t)__ldg(p.b_col + b0 + pj);
  const int64_t kp = p.dense ? pkp : (int64_t)__ldg(p.a_col + a0 + pkp);
  // Increment.
  long long v;
  if (p.integer) {
    // b_k'j != 0: the entry (j, k') of A under MAD_GRAM, else (k', j) of B.
    // The filter settles most tests with one load; the rest search rows.
    const unsigned long long ekey = (p.flags & MAD_GRAM)
                                        ? (((unsigned long long)j << 32) | (unsigned long long)kp)
                                        : (((unsigned long long)kp << 32) | (unsigned long long)j);
    bool hit = false;
    if (p.bloom && !bloom_may_contain(p.bloom, p.bloom_shift, ekey)) {
      hit = false;
    } else if (p.flags & MAD_GRAM) {
      const int64_t c0 = __ldg(p.b_ptr + kp), clen = __ldg(p.b_ptr + kp + 1) - c0;
      // B = A^T: b_k'j = a_jk'; search the shorter of the two sorted rows.
      const int64_t r0 = __ldg(p.a_ptr + j), rlen = __ldg(p.a_ptr + j + 1) - r0;
      hit = (rlen < clen) ? contains_sorted(p.a_col + r0, rlen, (int32_t)kp)
                          : contains_sorted(p.b_col + c0, clen, (int32_t)j);
    } else {
      const int64_t c0 = __ldg(p.b_ptr + kp), clen = __ldg(p.b_ptr + kp + 1) - c0;
      hit = contains_sorted(p.b_col + c0, clen, (int32_t)j);
    }
    v = hit ? 1 : 0;
  } else {
    const int64_t off = kp * p.ldb + j;
    const float b = p.b_f64 ? __double2float_rn(__ldg((const double*)p.b_val + off))
                            : __ldg((const float*)p.b_val + off);
    v = fixed_point(b, p.f_exp);
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

__device__ __forceinline__ Draw draw_one(const SampleParams& p, unsigned long long seed,
                                         unsigned long long ell, bool* bad) {
  const Uniforms u = diamond_uniforms(seed, ell);
  return draw_given_row(p, u, draw_row_i(p, u.u0, bad), bad);
}

}  // namespace mad

#endif  // MAD_DRAW_CUH_
