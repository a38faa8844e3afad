"""The bench's recall harness on CPU: the degree-pruned exact top-t of a
0/1 Gram product against the oracle's brute force, and the tie-aware
recall."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_degree_pruned_ground_truth_matches_bruteforce():
    import bench
    import oracle
    from paper_1506_03872_gb300.workloads import chung_lu
    w = chung_lu(nodes=1500, edges=15000, seed=21, t=30)
    M = oracle.Matrix(rowptr=w.rowptr, colidx=w.colidx, shape=(w.m, w.d))
    keys, c = oracle.Oracle(M, M, w.flags).bruteforce(w.t)
    tau, counts = bench.ground_truth_gram_binary(w.rowptr, w.colidx, w.t, "cpu", h0=64)
    assert tau == c[-1]
    i = (keys >> np.uint64(32)).astype(np.int64)
    j = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    got = counts(i, j)
    assert not np.isnan(got).any()        # every top pair lies inside the hub set
    assert np.array_equal(got, c)


def test_tie_aware_recall():
    import bench
    from paper_1506_03872_gb300.workloads import chung_lu
    w = chung_lu(nodes=1500, edges=15000, seed=21, t=30)
    tau, counts = bench.ground_truth_gram_binary(w.rowptr, w.colidx, w.t, "cpu", h0=64)
    gi = np.array([0, 1], dtype=np.uint32)
    gj = np.array([5, 9], dtype=np.uint32)
    gc = np.array([tau, tau - 1])
    r, _ = bench.recall_of(w, gi, gj, gc, set(), tau, counts)
    assert r == 1 / w.t
