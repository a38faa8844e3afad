"""Exact counts of 0/1 Gram candidates through mad_rescore (Alg. 3 on binary
inputs: c_ij is the number of columns rows i and j share) against numpy set
intersections, every candidate checked.  The grouped path (a shared-memory
bitmap of each hub's row) is taken with hubs whose candidates span several
units, diagonal pairs, equal degrees, empty rows and repeated pairs; the
per-pair merge path with more columns than that bitmap holds."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GRAM_EXCL = 2 | 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _transpose_csr(rowptr, colidx, m, d):
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rowptr))
    order = np.lexsort((rows, colidx))
    counts = np.bincount(colidx, minlength=d)
    rpt = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return rpt, rows[order].astype(np.int32)


def _expected(rowptr, colidx, i, j):
    out = np.empty(len(i), dtype=np.float64)
    for q, (a, b) in enumerate(zip(i.tolist(), j.tolist())):
        ra = colidx[rowptr[a]:rowptr[a + 1]]
        rb = colidx[rowptr[b]:rowptr[b + 1]]
        out[q] = len(np.intersect1d(ra, rb, assume_unique=True))
    return out


def _rescore_all(rowptr, colidx, shape, bt, i, j):
    """Every candidate's count from one mad_rescore call (t = all)."""
    import paper_1506_03872_gb300 as mad
    m, d = shape
    t = [torch.from_numpy(x).cuda() for x in (rowptr, colidx, bt[0], bt[1])]
    with mad.Context(GRAM_EXCL) as c:
        c.build(mad.csr(t[0], t[1], (m, d)), mad.csr(t[2], t[3], (d, m)), 1000, keep=tuple(t))
        cand = mad.encode_pairs(i, j)
        res, nr = mad.mad_rescore(c.ctx, cand, len(i), len(i))
        assert nr == len(i)
        gi, gj, _, gc = mad.decode_pairs(res, nr)
        assert mad.mad_stats(c.ctx)["device_error"] == 0
    return gi.astype(np.int64), gj.astype(np.int64), gc


def _check(rowptr, colidx, shape, bt, i, j):
    gi, gj, gc = _rescore_all(rowptr, colidx, shape, bt, i, j)
    want = _expected(rowptr, colidx, i, j)
    got = sorted(zip(gi.tolist(), gj.tolist(), gc.tolist()))
    exp = sorted(zip(i.tolist(), j.tolist(), want.tolist()))
    assert got == exp


def test_grouped_counts_exact():
    from paper_1506_03872_gb300 import workloads as W
    w = W.chung_lu(nodes=30000, edges=400000, seed=21)
    rowptr, colidx, m = w.rowptr, w.colidx, w.m
    deg = np.diff(rowptr)
    rng = _rng(22)
    hubs = np.argsort(-deg, kind="stable")[:40]
    pairs = []
    # Three hubs with 150 partners each: runs longer than a unit of 64.
    for h in hubs[:3]:
        for x in rng.choice(m, 150, replace=False):
            pairs.append((h, x))
    # Every pair among the 40 largest rows.
    for a in range(len(hubs)):
        for b in range(a + 1, len(hubs)):
            pairs.append((hubs[a], hubs[b]))
    # Diagonal pairs (c_ii = the row's length), of hubs and of short rows.
    for v in list(hubs[:5]) + list(rng.choice(m, 5, replace=False)):
        pairs.append((v, v))
    # Equal degrees: the hub is the smaller index.
    vals, first = np.unique(deg, return_index=True)
    for dv in vals[(vals > 2)][:10]:
        same = np.nonzero(deg == dv)[0][:3]
        if len(same) >= 2:
            pairs.append((same[0], same[1]))
            pairs.append((same[1], same[0]))
    # Empty rows, if the graph has any, against a hub and each other.
    empty = np.nonzero(deg == 0)[0][:2]
    for e in empty:
        pairs.append((e, hubs[0]))
    if len(empty) == 2:
        pairs.append((empty[0], empty[1]))
    # Random pairs, and some candidates twice.
    for _ in range(500):
        pairs.append(tuple(rng.integers(0, m, 2)))
    pairs += pairs[:20]
    p = np.array(pairs, dtype=np.int64)
    p = p[rng.permutation(len(p))]
    _check(rowptr, colidx, (m, m), (rowptr, colidx), p[:, 0], p[:, 1])


def test_grouped_counts_grow_between_calls():
    """A second, larger call on the same tables reallocates the grouping."""
    from paper_1506_03872_gb300 import workloads as W
    import paper_1506_03872_gb300 as mad
    w = W.chung_lu(nodes=8000, edges=80000, seed=23)
    rowptr, colidx, m = w.rowptr, w.colidx, w.m
    rng = _rng(24)
    t = [torch.from_numpy(x).cuda() for x in (rowptr, colidx)]
    with mad.Context(GRAM_EXCL) as c:
        A = mad.csr(t[0], t[1], (m, m))
        c.build(A, A, 1000, keep=tuple(t))
        for n in (100, 5000):
            i, j = rng.integers(0, m, n), rng.integers(0, m, n)
            res, nr = mad.mad_rescore(c.ctx, mad.encode_pairs(i, j), n, n)
            gi, gj, _, gc = mad.decode_pairs(res, nr)
            want = _expected(rowptr, colidx, i, j)
            assert sorted(zip(gi.tolist(), gj.tolist(), gc.tolist())) == \
                sorted(zip(i.tolist(), j.tolist(), want.tolist()))


def test_merge_path_counts_exact():
    """More columns (2^21) than the bitmap holds: the per-pair path."""
    rng = _rng(25)
    m, d = 2000, 1 << 21
    rows = []
    for r in range(m):
        k = int(rng.integers(0, 300)) if r % 50 else 0
        pop = rng.choice(5000, k // 2, replace=False)
        wide = rng.choice(d, k - k // 2, replace=False)
        rows.append(np.unique(np.concatenate([pop, wide])))
    rowptr = np.concatenate([[0], np.cumsum([len(x) for x in rows])]).astype(np.int64)
    colidx = np.concatenate(rows).astype(np.int32)
    bt = _transpose_csr(rowptr, colidx, m, d)
    i, j = rng.integers(0, m, 3000), rng.integers(0, m, 3000)
    i[:10] = j[:10]
    _check(rowptr, colidx, (m, d), bt, i, j)


def test_grouped_top_t_matches_oracle():
    """t < ncand: the top t by c (ties by smaller key), as the oracle's
    selection takes them, from counts that span several octaves."""
    import oracle
    import paper_1506_03872_gb300 as mad
    from paper_1506_03872_gb300 import workloads as W
    w = W.chung_lu(nodes=30000, edges=400000, seed=26)
    rowptr, colidx, m = w.rowptr, w.colidx, w.m
    deg = np.diff(rowptr)
    rng = _rng(27)
    hubs = np.argsort(-deg, kind="stable")[:120]
    pairs = {(int(min(a, b)), int(max(a, b))) for a in hubs for b in hubs if a != b}
    while len(pairs) < 12000:
        a, b = rng.integers(0, m, 2)
        if a != b:
            pairs.add((int(min(a, b)), int(max(a, b))))
    p = np.array(sorted(pairs), dtype=np.int64)
    p = p[rng.permutation(len(p))]
    i, j = p[:, 0], p[:, 1]
    keys = mad.keys_of(i.astype(np.uint32), j.astype(np.uint32))
    want = _expected(rowptr, colidx, i, j)
    t = [torch.from_numpy(x).cuda() for x in (rowptr, colidx)]
    with mad.Context(GRAM_EXCL) as c:
        A = mad.csr(t[0], t[1], (m, m))
        c.build(A, A, 1000, keep=tuple(t))
        for tt in (1, 300, 2048):
            res, nr = mad.mad_rescore(c.ctx, mad.encode_pairs(i, j), len(i), tt)
            gi, gj, _, gc = mad.decode_pairs(res, nr)
            tk, tc = oracle.topt(keys, want, tt)
            assert nr == len(tk)
            assert np.array_equal(mad.keys_of(gi, gj), tk)
            assert np.array_equal(gc, tc)
