"""The sharded protocol (paper_1506_03872_gb300/shard.py) on two gloo ranks
on the CPU.  Each rank's compute steps come from the oracle (its X over the
rank's diamond range) and plain sorts written here; the protocol itself --
contiguous diamond ranges, the all-to-all by key owner, the merge, the
owners' top t', the all-gather and the final selection and rescore -- is
the package's.  Omega_t' and Omega_t must equal one oracle run of all s
diamonds bit for bit."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _pairs(keys, xs, cs=None):
    """mad_pair records (n x 3 int64) from uint64 keys (i << 32 | j)."""
    keys = np.asarray(keys, dtype=np.uint64)
    raw = np.zeros((len(keys), 3), dtype=np.int64)
    i, j = keys >> np.uint64(32), keys & np.uint64(0xFFFFFFFF)
    raw[:, 0] = (i | (j << np.uint64(32))).view(np.int64)
    raw[:, 1] = np.asarray(xs, dtype=np.int64)
    if cs is not None:
        raw[:, 2] = np.asarray(cs, dtype=np.float64).view(np.int64)
    return torch.from_numpy(raw)


def _unpairs(p, n):
    raw = p[:n].numpy()
    w = raw[:, 0].view(np.uint64)
    keys = ((w & np.uint64(0xFFFFFFFF)) << np.uint64(32)) | (w >> np.uint64(32))
    return keys, raw[:, 1].copy(), raw[:, 2].copy().view(np.float64)


def _top(keys, xs, K):
    keep = xs > 0
    keys, xs = keys[keep], xs[keep]
    order = np.lexsort((keys, -xs))[:K]
    return keys[order], xs[order]


class OracleOps:
    """The compute steps on the CPU from the oracle (test only)."""

    def __init__(self, w):
        import oracle
        if w.csr:
            M = oracle.Matrix(rowptr=w.rowptr, colidx=w.colidx, shape=(w.m, w.d))
            self.o = oracle.Oracle(M, M, w.flags, w.s)
        else:
            self.o = oracle.Oracle(oracle.Matrix(w.A), oracle.Matrix(w.B), w.flags, w.s)
        self.acc = {}

    def sample(self, count, seed, first):
        self.o.reset()
        assert self.o.sample(count, seed, first) == 0

    def export_by_owner(self, world):
        keys, vals = self.o.x()
        owner = ((keys * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(40)) % np.uint64(world)
        order = np.argsort(owner, kind="stable")
        off = np.zeros(world + 1, dtype=np.int64)
        np.cumsum(np.bincount(owner.astype(np.int64), minlength=world), out=off[1:])
        return (torch.from_numpy(keys[order].view(np.int64).copy()),
                torch.from_numpy(vals[order].copy()), off)

    def reset(self):
        self.acc = {}

    def accumulate(self, keys, vals):
        for k, v in zip(keys.numpy().view(np.uint64).tolist(), vals.numpy().tolist()):
            self.acc[k] = self.acc.get(k, 0) + v

    def topk(self, tprime):
        keys = np.array(list(self.acc.keys()), dtype=np.uint64)
        xs = np.array(list(self.acc.values()), dtype=np.int64)
        k, x = _top(keys, xs, tprime)
        return _pairs(k, x), len(k)

    def select(self, pairs, n, K):
        keys, xs, _ = _unpairs(pairs, n)
        k, x = _top(keys, xs, K)
        return _pairs(k, x), len(k)

    def rescore(self, pairs, n, t):
        import oracle
        keys, xs, _ = _unpairs(pairs, n)
        c = self.o.rescore(keys)
        tk, tc = oracle.topt(keys, c, t)
        xmap = dict(zip(keys.tolist(), xs.tolist()))
        return _pairs(tk, [xmap[k] for k in tk.tolist()], tc), len(tk)


def _workload(name):
    from paper_1506_03872_gb300 import workloads as W
    if name == "plain_small":
        return W.plain_small(s=60_000)
    return W.chung_lu(nodes=3000, edges=30_000, seed=5, s=80_000, t=50, tprime=400)


def _rank_main(rank, world, port, name, outdir):
    import torch.distributed as dist

    from paper_1506_03872_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _workload(name)
        ops = OracleOps(w)
        res, n = shard.sharded_run(ops, dist, w.s, w.sampler_seed, w.tprime, w.t)
        np.save(os.path.join(outdir, f"res{rank}.npy"), res[:n].numpy())
        # The gathered Omega_t' as well (the input of the rescore).
        first, count = shard.diamond_range(w.s, rank, world)
        np.save(os.path.join(outdir, f"range{rank}.npy"), np.array([first, count]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("name", ["plain_small", "chung_lu_small"])
def test_two_gloo_ranks_equal_one_run(name, tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), name, str(tmp_path)), nprocs=world,
                       start_method="spawn")
    w = _workload(name)
    one = OracleOps(w).o
    keys, c = one.run(w.s, w.sampler_seed, w.tprime, w.t)
    ranges = [tuple(np.load(tmp_path / f"range{r}.npy")) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[0][1] + ranges[1][1] == w.s
    assert ranges[1][0] == ranges[0][1]
    for r in range(world):
        got = np.load(tmp_path / f"res{r}.npy")
        gk, gx, gc = _unpairs(torch.from_numpy(got), len(got))
        assert np.array_equal(gk, keys)
        assert np.array_equal(gc.view(np.int64), c.view(np.int64))


def test_diamond_ranges_cover_the_run():
    from paper_1506_03872_gb300.shard import diamond_range
    for s, world in ((10, 3), (1, 4), (10 ** 9 + 7, 8)):
        parts = [diamond_range(s, r, world) for r in range(world)]
        assert parts[0][0] == 0
        for (f0, c0), (f1, _) in zip(parts, parts[1:]):
            assert f0 + c0 == f1
        assert sum(c for _, c in parts) == s
