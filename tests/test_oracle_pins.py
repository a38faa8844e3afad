"""Pins of the CPU oracle to facts fixed outside it (no GPU).

Each test checks the oracle against something it cannot agree with by
construction: published Philox known-answer vectors, the paper's closed forms
(Lemma 1, Lemma 2, the binary diamond count c_ij^2 of Sec. 3.1), brute-force
products computed here with numpy, and long-double dot products.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import Matrix, Oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _w1_closed_form(A, B):
    """||W||_1 = sum_ik |a_ik| ||a_i*||_1 ||b_k*||_1 (Alg. 2 weight line)."""
    na = np.abs(A).sum(axis=1)
    nb = np.abs(B).sum(axis=1)
    return float((np.abs(A) * na[:, None] * nb[None, :]).sum())


def _dense(A, B, flags=0, s_max=1 << 20):
    return Oracle(Matrix(A), Matrix(B), flags=flags, s_max=s_max)


# ---------------------------------------------------------------------------
# Philox4x32-10
# ---------------------------------------------------------------------------
def test_philox_known_answers():
    rows = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            out = oracle.philox4x32_10(w[0:4], w[4:6])
            assert list(out) == w[6:10]
            rows += 1
    assert rows == 3


def test_diamond_uniforms_layout():
    # u0,u1 come from counter block 0, u2,u3 from block 1; word order lo|hi.
    seed, ell = 0x0123456789ABCDEF, (5 << 32) | 7
    u = oracle.diamond_uniforms(seed, ell)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    b0 = oracle.philox4x32_10([7, 5, 0, 0], key)
    b1 = oracle.philox4x32_10([7, 5, 0, 1], key)
    assert int(u[0]) == (int(b0[1]) << 32) | int(b0[0])
    assert int(u[1]) == (int(b0[3]) << 32) | int(b0[2])
    assert int(u[2]) == (int(b1[1]) << 32) | int(b1[0])
    assert int(u[3]) == (int(b1[3]) << 32) | int(b1[2])


def test_philox_uniformity():
    # 64-bit outputs: top byte uniform over 256 bins (chi-square).
    vals = np.array([oracle.diamond_uniforms(99, ell)[0] for ell in range(20000)], dtype=np.uint64)
    counts = np.bincount((vals >> np.uint64(56)).astype(np.int64), minlength=256)
    p = stats.chisquare(counts).pvalue
    assert p > 1e-4


# ---------------------------------------------------------------------------
# Norms and tables (Alg. 2 weight line, Sec. 4.2 cumulative tables)
# ---------------------------------------------------------------------------
def test_norms_match_exact_sums():
    rng = _rng(11)
    A = rng.standard_normal((40, 300)).astype(np.float32)
    B = rng.standard_normal((300, 700)).astype(np.float32)
    o = _dense(A, B)
    na = o.table("na").astype(np.float64)
    nb = o.table("nb").astype(np.float64)
    exact_a = np.abs(A.astype(np.float64)).sum(axis=1)
    exact_b = np.abs(B.astype(np.float64)).sum(axis=1)
    # FP32 error bound of 256 sequential partials + an 8-level tree.
    tol_a = (300 / 256 + 10) * 2.0 ** -24
    tol_b = (700 / 256 + 10) * 2.0 ** -24
    assert np.all(np.abs(na - exact_a) <= tol_a * exact_a)
    assert np.all(np.abs(nb - exact_b) <= tol_b * exact_b)


def _row_probs(prefix, ptr):
    out = []
    for r in range(len(ptr) - 1):
        seg = prefix[ptr[r]:ptr[r + 1]].astype(np.float64)
        q = np.diff(np.concatenate([[0.0], seg]))
        out.append(q / seg[-1] if len(seg) and seg[-1] > 0 else q)
    return out


def test_center_edge_law_equals_w_over_w1():
    """P(i,k) = (T1 step) x (T2 step) must equal w_ik / ||W||_1."""
    rng = _rng(12)
    A = rng.standard_normal((30, 20))
    B = rng.standard_normal((20, 50))
    o = _dense(A, B)
    T1 = o.table("T1").astype(np.float64)
    p_i = np.diff(np.concatenate([[0.0], T1])) / T1[-1]
    ptr = np.arange(0, 30 * 20 + 1, 20)
    p_k = np.array(_row_probs(o.table("T2"), ptr))
    joint = p_i[:, None] * p_k
    na = np.abs(A).sum(axis=1)
    nb = np.abs(B).sum(axis=1)
    w = np.abs(A) * na[:, None] * nb[None, :]
    ref = w / w.sum()
    assert np.max(np.abs(joint - ref) / ref) < 2e-5


def test_endpoint_laws():
    """j ~ |b_kj| / ||b_k*||_1 and k' ~ |a_ik'| / ||a_i*||_1."""
    rng = _rng(13)
    A = rng.standard_normal((25, 30)).astype(np.float32)
    B = rng.standard_normal((30, 40)).astype(np.float32)
    o = _dense(A, B)
    pa = np.array(_row_probs(o.table("TA"), np.arange(0, 25 * 30 + 1, 30)))
    pb = np.array(_row_probs(o.table("TB"), np.arange(0, 30 * 40 + 1, 40)))
    ra = np.abs(A.astype(np.float64))
    rb = np.abs(B.astype(np.float64))
    assert np.max(np.abs(pa - ra / ra.sum(1, keepdims=True))) < 2.0 ** -25
    assert np.max(np.abs(pb - rb / rb.sum(1, keepdims=True))) < 2.0 ** -25


def test_row_prefix_headroom():
    rng = _rng(14)
    A = (rng.standard_normal((10, 64)) * 1e30).astype(np.float32)
    B = (rng.standard_normal((64, 5000)) * 1e-30).astype(np.float32)
    o = _dense(A, B)
    for name in ("T2", "TA", "TB"):
        t = o.table(name)
        assert t.max() < 2 ** 31
        assert t.max() >= 2 ** 29  # scaled near the top of the range
    assert o.table("T1")[-1] < 2 ** 62


def test_zero_weights_never_drawn_and_bumped_weights_kept():
    A = np.array([[1.0, 0.0, 1e-30], [0.0, 0.0, 0.0], [2.0, -1.0, 0.0]])
    B = np.array([[1.0, 2.0], [0.0, -1.0], [3.0, 0.0]])
    o = _dense(A, B)
    T1 = o.table("T1")
    assert T1[1] == T1[0]  # the all-zero row of A is never a center
    T2 = o.table("T2")
    assert T2[1] == T2[0]  # a_01 = 0 gets no mass
    TA = o.table("TA")
    assert TA[2] - TA[1] == 1  # a_02 = 1e-30 is tiny but stays reachable
    assert o.scalars()["bumps"] >= 1
    i, k, j, kp, v = o.draw(5, 0, 20000)
    assert not np.any(i == 1)
    assert not np.any(A[i, k] == 0.0)
    assert not np.any(A[i, kp] == 0.0)
    assert not np.any(B[k, j] == 0.0)


def test_integer_tables_closed_form():
    """0/1 inputs: r_i = deg_i sum_{k in N(i)} deg_k; T2 = prefix of deg_k."""
    from paper_1506_03872_gb300.workloads import chung_lu
    w = chung_lu(nodes=300, edges=1500, seed=5)
    M = Matrix(rowptr=w.rowptr, colidx=w.colidx, shape=(w.m, w.d))
    o = Oracle(M, M, flags=w.flags)
    deg = np.diff(w.rowptr)
    r = np.array([deg[i] * deg[w.colidx[w.rowptr[i]:w.rowptr[i + 1]]].sum() for i in range(w.m)])
    assert np.array_equal(o.table("T1"), np.cumsum(r).astype(np.uint64))
    T2 = o.table("T2")
    TA = o.table("TA")
    for i in range(w.m):
        seg = slice(w.rowptr[i], w.rowptr[i + 1])
        assert np.array_equal(T2[seg], np.cumsum(deg[w.colidx[seg]]))
        assert np.array_equal(TA[seg], np.arange(1, deg[i] + 1))


# ---------------------------------------------------------------------------
# Lemma 1 and Lemma 2 (Sec. 5.1)
# ---------------------------------------------------------------------------
def _tiny_float():
    rng = _rng(21)
    A = rng.standard_normal((3, 2))
    B = rng.standard_normal((2, 3))
    return A, B


def test_lemma1_three_path_probability():
    A, B = _tiny_float()
    o = _dense(A, B)
    i, k, j, kp, prob, v = o.enumerate()
    w1 = _w1_closed_form(A, B)
    ref = np.abs(A[i, k] * B[k, j] * A[i, kp]) / w1
    assert len(i) == 3 * 2 * 3 * 2
    assert np.max(np.abs(prob - ref) / ref) < 1e-5
    assert abs(prob.sum() - 1.0) < 1e-12


def test_lemma2_expectation_dense():
    """E[x_ij / s] = c_ij^2 / ||W||_1 (x in units of 2^-F)."""
    rng = _rng(22)
    A = rng.standard_normal((4, 3))
    B = rng.standard_normal((3, 5))
    o = _dense(A, B)
    F = o.scalars()["F"]
    i, k, j, kp, prob, v = o.enumerate()
    ex = np.zeros((4, 5))
    np.add.at(ex, (i, j), prob * v.astype(np.float64) * 2.0 ** -F)
    C = A @ B
    ref = C ** 2 / _w1_closed_form(A, B)
    assert np.max(np.abs(ex - ref)) < 2e-5 * ref.max()


def test_lemma2_expectation_binary_exact():
    """0/1 inputs: every three-path has probability 1/||W||_1 and pair
    (i,j) closes exactly c_ij^2 of them (Sec. 3.1)."""
    rng = _rng(23)
    A = (rng.random((5, 4)) < 0.5).astype(np.int64)
    B = (rng.random((4, 6)) < 0.5).astype(np.int64)
    A[0, 0] = B[0, 0] = 1
    rpA = np.concatenate([[0], np.cumsum(A.sum(1))]).astype(np.int64)
    rpB = np.concatenate([[0], np.cumsum(B.sum(1))]).astype(np.int64)
    o = Oracle(Matrix(rowptr=rpA, colidx=np.nonzero(A)[1], shape=A.shape),
               Matrix(rowptr=rpB, colidx=np.nonzero(B)[1], shape=B.shape))
    i, k, j, kp, prob, v = o.enumerate()
    w1 = _w1_closed_form(A.astype(float), B.astype(float))
    assert np.allclose(prob * w1, 1.0, rtol=1e-12, atol=0)
    closed = np.zeros((5, 6), dtype=np.int64)
    np.add.at(closed, (i, j), v)
    C = A @ B
    assert np.array_equal(closed, C ** 2)
    # brute-force diamond count: (k, k') with a_ik b_kj a_ik' b_k'j = 1
    for ii in range(5):
        for jj in range(6):
            cnt = sum(A[ii, a] * B[a, jj] * A[ii, b] * B[b, jj] for a in range(4) for b in range(4))
            assert cnt == C[ii, jj] ** 2


def test_draw_frequencies_match_lemma1():
    """Chi-square of 200k oracle draws against the enumerated law."""
    A, B = _tiny_float()
    o = _dense(A, B)
    i, k, j, kp, prob, v = o.enumerate()
    index = {(a, b, c, d): q for q, (a, b, c, d) in enumerate(zip(i, k, j, kp))}
    di, dk, dj, dkp, dv = o.draw(seed=77, first=0, count=200_000)
    counts = np.zeros(len(prob))
    for q in zip(di, dk, dj, dkp):
        counts[index[tuple(int(x) for x in q)]] += 1
    exp = prob * len(di)
    small = exp < 5  # pool sparse bins so the chi-square approximation holds
    counts = np.concatenate([counts[~small], [counts[small].sum()]])
    exp = np.concatenate([exp[~small], [exp[small].sum()]])
    assert counts.sum() == len(di)
    p = stats.chisquare(counts, exp).pvalue
    assert p > 1e-4


def test_empirical_mean_within_5_sigma():
    A, B = _tiny_float()
    o = _dense(A, B, s_max=1 << 30)
    F = o.scalars()["F"]
    i, k, j, kp, prob, v = o.enumerate()
    mean = np.zeros((3, 3))
    second = np.zeros((3, 3))
    np.add.at(mean, (i, j), prob * v)
    np.add.at(second, (i, j), prob * v.astype(np.float64) ** 2)
    var = second - mean ** 2
    s, seeds = 4000, 40
    acc = np.zeros((3, 3))
    for seed in range(seeds):
        o.reset()
        assert o.sample(s, seed) == 0
        keys, vals = o.x()
        acc[(keys >> np.uint64(32)).astype(int), (keys & np.uint64(0xFFFFFFFF)).astype(int)] += vals
    emp = acc / seeds
    sigma = np.sqrt(s * var / seeds)
    assert np.all(np.abs(emp - s * mean) <= 5 * sigma + 1e-9 * 2.0 ** F)


# ---------------------------------------------------------------------------
# Postprocessing (Alg. 3) and ground truth
# ---------------------------------------------------------------------------
def test_bruteforce_matches_numpy():
    rng = _rng(31)
    A = rng.standard_normal((60, 8))
    B = rng.standard_normal((8, 70))
    o = _dense(A, B)
    keys, c = o.bruteforce(25)
    C = A @ B
    flat = np.abs(C).ravel()
    order = np.lexsort((np.arange(flat.size), -flat))[:25]
    ref_keys = (order // 70).astype(np.uint64) << np.uint64(32) | (order % 70).astype(np.uint64)
    assert np.array_equal(keys, ref_keys)
    assert np.allclose(c, C.ravel()[order], rtol=1e-14)


def test_rescore_dot_within_1e12_of_long_double():
    rng = _rng(32)
    A = rng.standard_normal((50, 300))
    B = rng.standard_normal((300, 40))
    o = _dense(A, B)
    ii, jj = np.meshgrid(np.arange(50), np.arange(40), indexing="ij")
    keys = (ii.ravel().astype(np.uint64) << np.uint64(32)) | jj.ravel().astype(np.uint64)
    c = o.rescore(keys)
    Al = A.astype(np.longdouble)
    Bl = B.astype(np.longdouble)
    ref = (Al[ii.ravel()] * Bl[:, jj.ravel()].T).sum(axis=1)
    scale = (np.abs(Al[ii.ravel()]) * np.abs(Bl[:, jj.ravel()].T)).sum(axis=1)
    err = np.abs(c.astype(np.longdouble) - ref)
    assert np.all(err <= 1e-12 * np.maximum(np.abs(ref), 1e-3 * scale))


def test_topk_order_and_ties():
    A = np.ones((4, 1))
    B = np.ones((1, 4))
    o = _dense(A, B, s_max=1 << 20)
    o.sample(4000, 3)
    keys, xs = o.topk(100)
    assert len(keys) == 16
    for q in range(len(keys) - 1):
        assert xs[q] > xs[q + 1] or (xs[q] == xs[q + 1] and keys[q] < keys[q + 1])
    allk, allx = o.x()
    assert set(keys.tolist()) == set(allk[allx > 0].tolist())


def test_topt_orders_by_abs_then_key():
    keys = np.array([5, 3, 9, 1], dtype=np.uint64)
    c = np.array([-2.0, 2.0, 1.0, -3.0])
    k, v = oracle.topt(keys, c, 3)
    assert k.tolist() == [1, 3, 5]
    assert v.tolist() == [-3.0, 2.0, -2.0]


def test_gram_keys_unordered_and_diagonal_skipped():
    from paper_1506_03872_gb300.workloads import chung_lu
    w = chung_lu(nodes=200, edges=1000, seed=6)
    M = Matrix(rowptr=w.rowptr, colidx=w.colidx, shape=(w.m, w.d))
    o = Oracle(M, M, flags=w.flags, s_max=1 << 20)
    o.sample(50_000, 1)
    keys, vals = o.x()
    i = keys >> np.uint64(32)
    j = keys & np.uint64(0xFFFFFFFF)
    assert np.all(i < j)
    sc = o.scalars()
    assert sc["diag_skipped"] > 0
    assert sc["inserted"] == vals.sum()


def test_planted_pairs_found_with_enough_samples():
    """With s well above ||W||_1 / tau^2 (Sec. 5.2) the top-t is exact."""
    from paper_1506_03872_gb300.workloads import plain_small
    w = plain_small(m=200, d=25, n=200, planted=10, seed=9)
    o = _dense(w.A, w.B, s_max=1 << 22)
    truth_keys, _ = o.bruteforce(10)
    keys, c = o.run(s=200_000, seed=4, tprime=100, t=10)
    assert set(keys.tolist()) == set(truth_keys.tolist())


def test_overflow_guard_on_s_max():
    A, B = _tiny_float()
    o = _dense(A, B, s_max=100)
    assert o.sample(60, 1) == 0
    assert o.sample(60, 1, 60) == 4  # overflow: more diamonds than s_max


def _sym_binary(n, p, seed):
    rng = _rng(seed)
    A = (rng.random((n, n)) < p).astype(np.int64)
    A = np.triu(A, 1)
    A = A + A.T
    A[0, 1] = A[1, 0] = 1
    rp = np.concatenate([[0], np.cumsum(A.sum(1))]).astype(np.int64)
    return A, Matrix(rowptr=rp, colidx=np.nonzero(A)[1], shape=A.shape)


def test_squared_symmetric_expectation_exact():
    """Sec. 3.2.3 on a symmetric 0/1 matrix: every closed three-path credits
    its pair {i, j} and its pair {k, k'}; the expected unordered-pair score
    per sample is 4 c_ab^2 / ||W||_1 for every off-diagonal pair (twice the
    Gram score 2 c_ab^2 / ||W||_1), from the enumerated law."""
    A, M = _sym_binary(6, 0.5, 31)
    flags = 2 | 4 | 8
    o = Oracle(M, M, flags)
    i, k, j, kp, prob, v = o.enumerate()
    w1 = _w1_closed_form(A.astype(float), A.astype(float))
    ex = np.zeros((6, 6))
    for a, b, pr, val in ((i, j, prob, v), (k, kp, prob, v)):
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        off = lo != hi
        np.add.at(ex, (lo[off], hi[off]), pr[off] * val[off])
    C = A @ A
    iu = np.triu_indices(6, 1)
    assert np.allclose(ex[iu] * w1, 4.0 * C[iu] ** 2, rtol=1e-12, atol=1e-12)


def test_squared_symmetric_expectation_dense():
    """Sec. 3.2.3 on a dense symmetric matrix with mixed signs: a diamond of
    (i, j) through (k, k') is one of (k, k') through (i, j) with the same
    sign product, so the unordered-pair score per sample is again
    4 c_ab^2 / ||W||_1 (x in units of 2^-F), up to the tables' rounding."""
    rng = _rng(34)
    S = rng.standard_normal((5, 5))
    S = S + S.T
    S[1, 3] = S[3, 1] = 0.0
    o = _dense(S, S.copy(), flags=2 | 4 | 8)
    F = o.scalars()["F"]
    i, k, j, kp, prob, v = o.enumerate()
    ex = np.zeros((5, 5))
    for a, b in ((i, j), (k, kp)):
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        off = lo != hi
        np.add.at(ex, (lo[off], hi[off]), prob[off] * v[off].astype(np.float64) * 2.0 ** -F)
    C = S @ S
    iu = np.triu_indices(5, 1)
    ref = 4.0 * C[iu] ** 2 / _w1_closed_form(S, S)
    assert np.max(np.abs(ex[iu] - ref)) < 2e-5 * ref.max()
    assert np.all(ex[np.tril_indices(5)] == 0.0)


def test_squared_symmetric_counts_and_flag_rule():
    """One draw of the sampler adds to at most two pairs: X from sampling
    equals the sum over the drawn diamonds of the two additions (checked
    against the diamonds the oracle reports), and the flag needs Gram
    inputs."""
    A, M = _sym_binary(40, 0.15, 32)
    o = Oracle(M, M, 2 | 4 | 8, 5000)
    assert o.sample(5000, 9) == 0
    keys, vals = o.x()
    di, dk, dj, dkp, dv = o.draw(seed=9, first=0, count=5000)
    ref = {}
    for a, b, c, e, val in zip(di, dk, dj, dkp, dv):
        for p_, q_ in ((a, c), (b, e)):
            if p_ == q_ or val == 0:
                continue
            key = (int(min(p_, q_)) << 32) | int(max(p_, q_))
            ref[key] = ref.get(key, 0) + int(val)
    got = {int(kk): int(vv) for kk, vv in zip(keys, vals)}
    assert got == ref
    with pytest.raises(Exception):
        Oracle(M, M, 8)


def test_mlp_reference_gradient_matches_finite_differences():
    """The NumPy statement of the budget perceptron: its backward pass is the
    derivative of its loss (unrounded weights, float64, smooth region)."""
    import mlp_reference as R
    rng = _rng(33)
    f, n = 5, 40
    p = rng.standard_normal(R.H * f + 3 * R.H + R.H * R.H + 1) * 0.2
    X = rng.standard_normal((n, f))
    y = rng.standard_normal(n) * 3
    loss, g = R.loss_and_grad(p, X, y, 0.8, np.float64, round_weights=False)
    idx = rng.choice(len(p), 40, replace=False)
    for q in idx:
        e = np.zeros_like(p)
        e[q] = 1e-6
        lp, _ = R.loss_and_grad(p + e, X, y, 0.8, np.float64, round_weights=False)
        lm, _ = R.loss_and_grad(p - e, X, y, 0.8, np.float64, round_weights=False)
        assert abs((lp - lm) / 2e-6 - g[q]) < 1e-5 * max(1.0, abs(g[q]))


def test_bf16_rounding_reference():
    """BF16 round-to-nearest-even of the reference against the exact rule
    on hand-picked halfway cases."""
    import mlp_reference as R
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7, -2.5], np.float32)
    assert np.array_equal(R.bf16(x), np.array([1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, -2.5],
                                              np.float32))


# ---------------------------------------------------------------------------
# 0/1 inputs: exact counts (Alg. 3 on binary inputs; c_ij counts the common
# entries, Sec. 3.1) and the exact sparse product (Sec. 4.3)
# ---------------------------------------------------------------------------
def _csr_of(D):
    """CSR (rowptr, colidx) of a 0/1 numpy matrix (columns ascending)."""
    rp = np.concatenate([[0], np.cumsum((D != 0).sum(1))]).astype(np.int64)
    return Matrix(rowptr=rp, colidx=np.nonzero(D)[1].astype(np.int32), shape=D.shape)


def _uneven_binary(m, d, seed):
    """0/1 matrix whose rows have very uneven degrees: row r keeps each
    entry with probability 0.9^r-ish, plus a few full and empty rows."""
    rng = _rng(seed)
    p = 0.9 ** (np.arange(m) % 40)[:, None] * np.ones((1, d))
    D = (rng.random((m, d)) < p).astype(np.int64)
    D[3] = 1          # a full row
    D[5] = 0          # an empty row
    return D


def _ref_topt(C, t, gram=False, exclude_diag=False, stored=None):
    """numpy top-t of |C| by (|c| desc, key asc) under the pair rules."""
    m, n = C.shape
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    keep = np.ones(C.shape, bool)
    if gram:
        keep &= jj >= ii
    if exclude_diag:
        keep &= jj != ii
    if stored is not None:
        keep &= stored
    i, j, c = ii[keep], jj[keep], C[keep]
    order = np.lexsort((j, i, -np.abs(c)))[:t]
    keys = (i[order].astype(np.uint64) << np.uint64(32)) | j[order].astype(np.uint64)
    return keys, c[order].astype(np.float64)


def test_binary_rescore_counts_match_numpy_bipartite():
    """Oracle.rescore on 0/1 CSR inputs with A != B^T equals (A B)_ij."""
    A = _uneven_binary(70, 50, 41)
    B = (_rng(42).random((50, 90)) < 0.2).astype(np.int64)
    B[:, 7] = 1       # a full column
    o = Oracle(_csr_of(A), _csr_of(B), 0)
    ii, jj = np.meshgrid(np.arange(70), np.arange(90), indexing="ij")
    keys = (ii.ravel().astype(np.uint64) << np.uint64(32)) | jj.ravel().astype(np.uint64)
    c = o.rescore(keys)
    assert np.array_equal(c, (A @ B)[ii.ravel(), jj.ravel()].astype(np.float64))


def test_binary_rescore_counts_match_numpy_gram_with_diagonal():
    """Gram inputs (A = B^T, here a symmetric adjacency of uneven degrees):
    every pair including i == j equals (A A^T)_ij = |N(i) ∩ N(j)|."""
    D = _uneven_binary(60, 60, 43)
    S = np.triu(D, 1)
    S = S + S.T
    M = _csr_of(S)
    o = Oracle(M, M, 2)
    ii, jj = np.meshgrid(np.arange(60), np.arange(60), indexing="ij")
    up = jj >= ii
    keys = (ii[up].astype(np.uint64) << np.uint64(32)) | jj[up].astype(np.uint64)
    c = o.rescore(keys)
    assert np.array_equal(c, (S @ S.T)[ii[up], jj[up]].astype(np.float64))
    assert np.array_equal(c[ii[up] == jj[up]], S.sum(1).astype(np.float64))  # c_ii = deg


def test_binary_bruteforce_matches_numpy_with_ties():
    """or_bruteforce on 0/1 CSR inputs (bipartite, Gram, Gram without the
    diagonal) equals numpy's top t of A B, ties broken by the smaller key;
    counts of small integers tie often."""
    A = _uneven_binary(50, 30, 44)
    B = (_rng(45).random((30, 40)) < 0.3).astype(np.int64)
    keys, c = Oracle(_csr_of(A), _csr_of(B), 0).bruteforce(60)
    rk, rc = _ref_topt(A @ B, 60)
    assert np.array_equal(keys, rk) and np.array_equal(c, rc)
    assert len(np.unique(rc)) < len(rc)        # the case has ties
    S = np.triu(_uneven_binary(45, 45, 46), 1)
    S = S + S.T
    M = _csr_of(S)
    for flags, ex in ((2, False), (2 | 4, True)):
        keys, c = Oracle(M, M, flags).bruteforce(80)
        rk, rc = _ref_topt(S @ S, 80, gram=True, exclude_diag=ex)
        assert np.array_equal(keys, rk) and np.array_equal(c, rc)


def test_sparse_exact_matches_numpy_and_bruteforce():
    """The row-wise sparse product (Sec. 4.3) gives numpy's top t over the
    stored entries of C (pairs some k reaches), ties by key, and the brute
    force's top t whenever t stored entries exist."""
    A = _uneven_binary(50, 30, 47)
    B = (_rng(48).random((30, 40)) < 0.3).astype(np.int64)
    o = Oracle(_csr_of(A), _csr_of(B), 0)
    C = A @ B
    for t in (1, 37, 200):
        keys, c = o.sparse_exact(t)
        rk, rc = _ref_topt(C, t, stored=C != 0)
        assert np.array_equal(keys, rk) and np.array_equal(c, rc)
        bk, bc = o.bruteforce(t)
        assert np.array_equal(keys, bk) and np.array_equal(c, bc)
    S = np.triu(_uneven_binary(45, 45, 49), 1)
    S = S + S.T
    M = _csr_of(S)
    for flags, ex in ((2, False), (2 | 4, True)):
        o = Oracle(M, M, flags)
        keys, c = o.sparse_exact(90)
        rk, rc = _ref_topt(S @ S, 90, gram=True, exclude_diag=ex, stored=(S @ S) != 0)
        assert np.array_equal(keys, rk) and np.array_equal(c, rc)
    # Fewer stored entries than t: only the stored ones are returned.
    E = np.zeros((6, 5), np.int64)
    E[1, 2] = E[4, 0] = 1
    F = np.zeros((5, 7), np.int64)
    F[2, 3] = F[0, 3] = F[0, 6] = 1
    keys, c = Oracle(_csr_of(E), _csr_of(F), 0).sparse_exact(10)
    assert keys.tolist() == [(1 << 32) | 3, (4 << 32) | 3, (4 << 32) | 6]
    assert c.tolist() == [1.0, 1.0, 1.0]


# ---------------------------------------------------------------------------
# Wedge sampling (the appendix's Alg. "MAD wedge sampling" and its Lemmas)
# ---------------------------------------------------------------------------
def _wedge_w1(A, B):
    """||w||_1 = sum_k ||a_*k||_1 ||b_k*||_1 (the wedge weights)."""
    return float((np.abs(A).sum(axis=0) * np.abs(B).sum(axis=1)).sum())


def test_wedge_expectation_dense():
    """Enumerated wedge law: every wedge (i,k,j) has probability
    |a_ik||b_kj| / ||w||_1 and E[x_ij]/s = c_ij / ||w||_1 (up to the
    tables' fixed-point rounding)."""
    rng = _rng(51)
    A = rng.standard_normal((5, 4))
    B = rng.standard_normal((4, 6))
    A[1, 2] = 0.0
    o = Oracle(Matrix(A), Matrix(B), oracle.WEDGE)
    i, k, j, prob, v = o.enumerate_wedges()
    w1 = _wedge_w1(A, B)
    assert abs(prob.sum() - 1.0) < 1e-12
    assert np.allclose(prob, np.abs(A[i, k] * B[k, j]) / w1, rtol=2e-5)
    assert np.array_equal(v, np.sign(A[i, k] * B[k, j]).astype(np.int64))
    ex = np.zeros((5, 6))
    np.add.at(ex, (i, j), prob * v)
    C = A @ B
    assert np.allclose(ex * w1, C, atol=2e-5 * np.abs(C).max())


def test_wedge_expectation_binary_exact():
    """0/1 inputs: every wedge has probability exactly 1 / ||w||_1 and the
    pair (i, j) is reached by exactly c_ij wedges, so E[x_ij]/s =
    c_ij / ||w||_1 holds exactly."""
    rng = _rng(52)
    A = (rng.random((7, 5)) < 0.5).astype(np.int64)
    B = (rng.random((5, 8)) < 0.5).astype(np.int64)
    A[0, 0] = B[0, 0] = 1
    o = Oracle(_csr_of(A), _csr_of(B), oracle.WEDGE)
    i, k, j, prob, v = o.enumerate_wedges()
    w1 = int((A.sum(axis=0) * B.sum(axis=1)).sum())
    assert len(prob) == w1
    assert np.all(prob * w1 == 1.0) and np.all(v == 1)
    cnt = np.zeros((7, 8), np.int64)
    np.add.at(cnt, (i, j), 1)
    assert np.array_equal(cnt, A @ B)
    assert int(o.table("TK")[-1]) == w1


def test_wedge_draw_frequencies_match_the_law():
    rng = _rng(53)
    A = np.abs(rng.standard_normal((4, 3))) + 0.1
    B = rng.standard_normal((3, 5))
    o = Oracle(Matrix(A), Matrix(B), oracle.WEDGE, 1 << 20)
    i, k, j, prob, _ = o.enumerate_wedges()
    n = 200_000
    di, dk, dj, dkp, dv = o.draw(seed=7, first=0, count=n)
    assert np.all(dkp == 0)
    idx = {(a, b, c): q for q, (a, b, c) in enumerate(zip(i.tolist(), k.tolist(), j.tolist()))}
    counts = np.zeros(len(prob))
    for a, b, c in zip(di.tolist(), dk.tolist(), dj.tolist()):
        counts[idx[(a, b, c)]] += 1
    p = stats.chisquare(counts, prob * n).pvalue
    assert p > 1e-4


def test_wedge_sample_accumulates_its_draws_with_pair_rules():
    """X after s wedges is the sum of the drawn increments on the keys of
    the pair rules (Gram: unordered, diagonal skipped and counted)."""
    A, M = _sym_binary(30, 0.2, 54)
    o = Oracle(M, M, 2 | 4 | oracle.WEDGE, 20_000)
    assert o.sample(20_000, 5) == 0
    keys, vals = o.x()
    di, dk, dj, _, dv = o.draw(seed=5, first=0, count=20_000)
    ref, diag = {}, 0
    for a, c, val in zip(di.tolist(), dj.tolist(), dv.tolist()):
        if a == c:
            diag += 1
            continue
        key = (min(a, c) << 32) | max(a, c)
        ref[key] = ref.get(key, 0) + val
    assert {int(k_): int(v_) for k_, v_ in zip(keys, vals)} == ref
    assert o.scalars()["diag_skipped"] == diag


def test_wedge_sampling_finds_planted_pairs():
    from paper_1506_03872_gb300.workloads import plain_small
    w = plain_small(m=200, d=25, n=200, planted=10, seed=9)
    o = Oracle(Matrix(w.A), Matrix(w.B), oracle.WEDGE, 1 << 22)
    truth, _ = o.bruteforce(10)
    keys, c = o.run(s=2_000_000, seed=4, tprime=100, t=10)
    assert set(keys.tolist()) == set(truth.tolist())


# ---------------------------------------------------------------------------
# Alias tables (Sec. 4.1: the alias method for constant-time draws)
# ---------------------------------------------------------------------------
def _alias_instance(seed=71, m=1500, d=7, n=2500):
    """T1 over 1500 rows and TB rows of 2500 entries have two levels
    (segments of 1024 entries); the rows of T2 and TA have one.  A few exact
    zeros give zero weights."""
    rng = _rng(seed)
    A = rng.standard_normal((m, d)) * np.exp(0.7 * rng.standard_normal((m, 1)))
    B = rng.standard_normal((d, n)) * np.exp(0.7 * rng.standard_normal((1, n)))
    A[rng.random(A.shape) < 0.03] = 0.0
    B[:, 5] = 0.0
    return A, B


def _weights(prefix, L):
    """Per-row weights of a prefix table with rows of length L."""
    P = prefix.astype(np.int64).reshape(-1, L)
    return np.diff(np.concatenate([np.zeros((P.shape[0], 1), np.int64), P], axis=1), axis=1)


def _check_alias_level(ent, x):
    """One alias table over integer weights x: n x_i equals the mass that the
    table sends to i, t_c for its own column plus X - t_c from every column
    whose alias it is; thresholds in [0, X], aliases in range."""
    n = len(x)
    X = int(sum(int(v) for v in x))
    t = [int(v) for v in ent["t"]]
    a = [int(v) for v in ent["a"]]
    assert all(0 <= v <= X for v in t) and all(0 <= v < n for v in a)
    mass = [0] * n
    for c in range(n):
        mass[c] += t[c]
        mass[a[c]] += X - t[c]
    assert mass == [n * int(v) for v in x]


def test_alias_tables_reproduce_the_weights_exactly():
    """Every level of every alias table (T1 and TB with two levels, T2 and
    TA with one) gives each entry exactly its weight over the total, in
    integers: P(c) = x_c / X."""
    A, B = _alias_instance()
    o = _dense(A, B, flags=oracle.ALIAS)
    m, d = A.shape
    n = B.shape[1]
    fams = {"T1": _weights(o.table("T1"), m), "T2": _weights(o.table("T2"), d),
            "TA": _weights(o.table("TA"), d), "TB": _weights(o.table("TB"), n)}
    S = oracle.ALIAS_SEG
    for name, W in fams.items():
        ent, segX, rowX = o.alias_table(name)
        rows, L = W.shape
        nseg = (L + S - 1) // S
        assert len(ent) == rows * (L + nseg) and len(segX) == rows * nseg
        for r in range(rows) if rows < 50 else [0, 1, rows // 2, rows - 1]:
            e = ent[r * (L + nseg):(r + 1) * (L + nseg)]
            seg = []
            for s in range(nseg):
                x = W[r, s * S:(s + 1) * S]
                assert int(segX[r * nseg + s]) == int(x.sum())
                _check_alias_level(e[s * S:s * S + len(x)], x)
                seg.append(int(x.sum()))
            assert int(rowX[r]) == int(W[r].sum())
            if nseg > 1:
                _check_alias_level(e[L:], seg)


def _chi2_pvalue(obs, p):
    from scipy.stats import chisquare
    keep = p > 0
    assert obs[~keep].sum() == 0   # never drawn where the law is 0
    return chisquare(obs[keep], p[keep] * obs.sum()).pvalue


def test_alias_draws_follow_the_laws():
    """The alias draw mapping: 400k diamonds of the alias sampler.  Row i
    (two-level T1) and column j (two-level TB rows, through the marginal over
    k) against their exact laws by chi-square; zero-weight entries never
    drawn."""
    A, B = _alias_instance()
    o = _dense(A, B, flags=oracle.ALIAS)
    m, d = A.shape
    n = B.shape[1]
    i, k, j, kp, v = o.draw(seed=5, first=1 << 20, count=400_000)
    w1 = _weights(o.table("T1"), m)[0].astype(np.float64)
    p_i = w1 / w1.sum()
    assert _chi2_pvalue(np.bincount(i, minlength=m).astype(float), p_i) > 1e-4
    # j's marginal: sum_k P(k) P(j | k), P(k) from the T2 rows of the drawn i.
    T2w = _weights(o.table("T2"), d).astype(np.float64)
    TBw = _weights(o.table("TB"), n).astype(np.float64)
    pk_given_i = T2w / T2w.sum(axis=1, keepdims=True)
    p_k = p_i @ pk_given_i
    p_j = p_k @ (TBw / TBw.sum(axis=1, keepdims=True))
    assert _chi2_pvalue(np.bincount(j, minlength=n).astype(float), p_j) > 1e-4
    assert not np.any(j == 5)   # column 5 of B is zero: weight 0 in every TB row


def test_alias_joint_law_on_a_tiny_instance():
    """All four draws at once on an instance small enough to enumerate: the
    alias sampler's (i, k, j, k') frequencies against the enumerated law of
    Lemma 1 (the same law as the prefix-table sampler's)."""
    rng = _rng(72)
    A = rng.standard_normal((4, 3))
    B = rng.standard_normal((3, 5))
    A[1, 2] = 0.0
    o = _dense(A, B, flags=oracle.ALIAS)
    ei, ek, ej, ekp, prob, _ = _dense(A, B).enumerate()
    idx = {(a, b, c, e): q for q, (a, b, c, e) in enumerate(zip(ei, ek, ej, ekp))}
    i, k, j, kp, _ = o.draw(seed=9, first=0, count=300_000)
    obs = np.zeros(len(prob))
    for t in zip(i, k, j, kp):
        obs[idx[t]] += 1
    assert _chi2_pvalue(obs, prob) > 1e-4


def test_alias_flag_rules():
    """Alias tables are built for dense float inputs: 0/1 inputs and wedge
    sampling refuse the flag."""
    A, M = _sym_binary(20, 0.2, 73)
    with pytest.raises(Exception):
        Oracle(M, M, oracle.ALIAS | 2)
    rng = _rng(74)
    with pytest.raises(Exception):
        _dense(rng.standard_normal((5, 3)), rng.standard_normal((3, 4)),
               flags=oracle.ALIAS | oracle.WEDGE)
