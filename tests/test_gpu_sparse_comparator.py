"""The exact comparator for 0/1 inputs (Sec. 4.3) on the GPU, through the C
ABI, against the oracle's row-wise sparse product: the same pairs in the
same order and the same integer counts, bit for bit, ties included."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _csr(D):
    rp = np.concatenate([[0], np.cumsum((D != 0).sum(1))]).astype(np.int64)
    return rp, np.nonzero(D)[1].astype(np.int32)


def _run(rpA, ciA, shapeA, rpB, ciB, shapeB, flags, t, options=0):
    import oracle
    import paper_1506_03872_gb300 as mad
    tA = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (rpA, ciA)]
    tB = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (rpB, ciB)]
    with mad.Context(flags) as c:
        out, n = mad.mad_sparse_topt(c.ctx, mad.csr(tA[0], tA[1], shapeA),
                                     mad.csr(tB[0], tB[1], shapeB), t, options)
        gi, gj, gx, gc = mad.decode_pairs(out, n)
    MA = oracle.Matrix(rowptr=rpA, colidx=ciA, shape=shapeA)
    MB = oracle.Matrix(rowptr=rpB, colidx=ciB, shape=shapeB)
    keys, c = oracle.Oracle(MA, MB, flags).sparse_exact(t)
    got = (gi.astype(np.uint64) << np.uint64(32)) | gj.astype(np.uint64)
    return got, gc, gx, keys, c


def _check(got, gc, gx, keys, c):
    assert len(got) == len(keys)
    assert np.array_equal(got, keys)
    assert np.array_equal(gc, c)
    assert np.all(gx == 0)


@pytest.mark.parametrize("nodes,edges,t", [(10_000, 100_000, 100), (10_000, 100_000, 1000),
                                           (100_000, 1_000_000, 1000)])
@pytest.mark.parametrize("options", [0, 1])
def test_chung_lu_gram_matches_oracle(nodes, edges, t, options):
    """Common-neighbour counts of Chung-Lu graphs (unordered pairs, diagonal
    excluded): the degree-bounded pass and the pass over every row."""
    from paper_1506_03872_gb300.workloads import chung_lu
    if options and nodes > 10_000:
        pytest.skip("every-row pass checked on the smaller graphs")
    w = chung_lu(nodes=nodes, edges=edges, seed=71 + nodes % 97, t=t)
    shape = (w.m, w.d)
    _check(*_run(w.rowptr, w.colidx, shape, w.rowptr, w.colidx, shape, w.flags, t, options))


def test_many_windows_without_bound():
    """More selected columns than one shared window holds (labels in
    several windows, Gram rows starting inside a later window)."""
    from paper_1506_03872_gb300.workloads import chung_lu
    w = chung_lu(nodes=60_000, edges=240_000, seed=77, t=300)
    shape = (w.m, w.d)
    _check(*_run(w.rowptr, w.colidx, shape, w.rowptr, w.colidx, shape, w.flags, 300, 1))


@pytest.mark.parametrize("flags", [0, 4])
def test_bipartite_matches_oracle(flags):
    """A != B^T with rows and columns of uneven degree; with flag 4 the pairs
    i == j are excluded."""
    rng = _rng(81)
    p_row = 0.3 * 0.93 ** (np.arange(700) % 50)
    A = (rng.random((700, 400)) < p_row[:, None]).astype(np.int64)
    A[5] = 0
    B = (rng.random((400, 900)) < 0.05).astype(np.int64)
    B[:, 11] = 1
    B[:, 12] = 0
    rpA, ciA = _csr(A)
    rpB, ciB = _csr(B)
    _check(*_run(rpA, ciA, A.shape, rpB, ciB, B.shape, flags, 500))


def test_gram_with_diagonal():
    """Gram pairs with the diagonal kept: c_ii = deg_i competes."""
    from paper_1506_03872_gb300.workloads import chung_lu
    w = chung_lu(nodes=5000, edges=40_000, seed=83, t=200)
    shape = (w.m, w.d)
    _check(*_run(w.rowptr, w.colidx, shape, w.rowptr, w.colidx, shape, 2, 200))


@pytest.mark.parametrize("flags,t", [(2 | 4, 1000), (2 | 4, 500_000), (2, 1000), (0, 3000)])
def test_ties_beyond_the_candidate_list(flags, t):
    """Every pair of leaves of a star shares the centre (c = 1, about 1.1e6
    tied pairs), and every entry of a rank-one all-ones product ties: more
    tied candidates than the list holds, so the pass takes the exact
    histogram threshold and the smallest keys among the ties."""
    if flags:
        n = 1500
        D = np.zeros((n, n), np.int64)
        D[0, 1:] = D[1:, 0] = 1
        rp, ci = _csr(D)
        _check(*_run(rp, ci, D.shape, rp, ci, D.shape, flags, t))
    else:
        A = np.ones((1100, 1), np.int64)
        B = np.ones((1, 1000), np.int64)
        rpA, ciA = _csr(A)
        rpB, ciB = _csr(B)
        _check(*_run(rpA, ciA, A.shape, rpB, ciB, B.shape, flags, t))


def test_fewer_stored_entries_than_t():
    A = np.zeros((6, 5), np.int64)
    A[1, 2] = A[4, 0] = 1
    B = np.zeros((5, 7), np.int64)
    B[2, 3] = B[0, 3] = B[0, 6] = 1
    rpA, ciA = _csr(A)
    rpB, ciB = _csr(B)
    got, gc, gx, keys, c = _run(rpA, ciA, A.shape, rpB, ciB, B.shape, 0, 10)
    _check(got, gc, gx, keys, c)
    assert len(got) == 3


def test_zero_product_and_errors():
    """C = 0 (A's columns meet only empty rows of B) returns no pair; other
    formats and bad shapes are refused."""
    import paper_1506_03872_gb300 as mad
    A = np.zeros((4, 3), np.int64)
    A[:, 0] = 1
    B = np.zeros((3, 5), np.int64)
    B[1, 2] = 1
    rpA, ciA = _csr(A)
    rpB, ciB = _csr(B)
    tA = [torch.from_numpy(x).cuda() for x in (rpA, ciA)]
    tB = [torch.from_numpy(x).cuda() for x in (rpB, ciB)]
    MA, MB = mad.csr(tA[0], tA[1], (4, 3)), mad.csr(tB[0], tB[1], (3, 5))
    with mad.Context() as c:
        _, n = mad.mad_sparse_topt(c.ctx, MA, MB, 5)
        assert n == 0
        with pytest.raises(mad.MadError) as e:
            mad.mad_sparse_topt(c.ctx, MA, MB, 0)
        assert e.value.status == 1
        with pytest.raises(mad.MadError) as e:
            mad.mad_sparse_topt(c.ctx, MA, mad.csr(tA[0], tA[1], (4, 3)), 5)
        assert e.value.status == 1
        dense = torch.ones(4, 3, device="cuda")
        with pytest.raises(mad.MadError) as e:
            mad.mad_sparse_topt(c.ctx, mad.dense(dense), MB, 5)
        assert e.value.status == 8
        with pytest.raises(mad.MadError) as e:
            mad.mad_sparse_topt(c.ctx, MA, MB, 5, options=2)
        assert e.value.status == 1
