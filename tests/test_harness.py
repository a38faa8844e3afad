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


def test_reference_arm_line_on_cpu():
    """bench.py --impl reference times the CPU oracle and prints one JSON
    line with the contract's keys (no GPU needed)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--scale", "0.02",
                          "--cpu-diamonds", "100000"],
                         capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "diamonds/s"
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == "dense_factors"
    assert line["config"]["l2"] and line["config"]["parallelism"] == "single"
    assert "200000 of the 200000 diamonds" in line["cpu_baseline"]["sample"]


def test_all_core_oracle_merge_equals_one_core():
    """The CPU baseline's all-cores leg: contiguous diamond ranges sampled by
    one oracle each merge to the X of one oracle over the whole range."""
    import bench
    from paper_1506_03872_gb300.workloads import dense_factors
    w = dense_factors(m=3000, n=800, s=60_000)
    res = bench.cpu_baseline(w, 60_000, threads=3)
    assert res["all_cores"]["merged_x_equals_one_core"] is True
    assert res["cores"] == 3 and res["all_cores"]["diamonds"] == 60_000
    assert res["one_core"]["diamonds_per_s"] > 0 and res["cpu_model"]
