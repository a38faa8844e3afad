"""The library steps of a sharded run (mad_export_x_by_owner,
mad_accumulate, mad_select_pairs) on one GPU, with the ranks emulated one
after another in one process (no collective: the owner segments are handed
over here): the partial X of the diamond ranges, merged by owner, equal the
X of one context that sampled every diamond, and Omega_t' and Omega_t equal
that context's and the oracle's bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from gpu_cases import Case  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _x_sorted(mad, ctx, cap):
    keys, vals, n = mad.mad_export_x(ctx, cap=cap)
    k = keys[:n].cpu().numpy().view(np.uint64)
    v = vals[:n].cpu().numpy()
    order = np.argsort(k)
    return k[order], v[order]


@pytest.mark.parametrize("name,world", [("dense_ragged_f32", 2), ("dense_factors_small", 3),
                                        ("chung_lu_small", 2), ("bipartite_binary", 4)])
def test_emulated_ranks_equal_one_run(name, world):
    import paper_1506_03872_gb300 as mad
    from paper_1506_03872_gb300.shard import LibraryOps, diamond_range
    s, seed, tprime, t = 240_000, 31, 1500, 40
    ranks = [Case(name, s_max=s) for _ in range(world)]
    one = Case(name, s_max=s)
    try:
        ops = [LibraryOps(c.ctx.ctx, export_cap=1 << 12) for c in ranks]
        for r in range(world):
            first, count = diamond_range(s, r, world)
            ops[r].sample(count, seed, first)
        parts = [ops[r].export_by_owner(world) for r in range(world)]
        # every partial key goes to exactly one owner
        total = sum(int(p[2][-1]) for p in parts)
        assert total == sum(len(_x_sorted(mad, c.ctx.ctx, s + 1)[0]) for c in ranks)
        cands = []
        for o in range(world):
            rk = torch.cat([k[int(off[o]):int(off[o + 1])] for k, _, off in parts])
            rv = torch.cat([v[int(off[o]):int(off[o + 1])] for _, v, off in parts])
            ops[o].reset()
            ops[o].accumulate(rk, rv)
            cand, nc = ops[o].topk(tprime)
            cands.append(cand[:nc])
        # The owners' X together are the one-run X, key for key.
        mad.mad_sample(one.ctx.ctx, s, seed)
        ok, ov = _x_sorted(mad, one.ctx.ctx, s + 1)
        merged = [_x_sorted(mad, c.ctx.ctx, s + 1) for c in ranks]
        mk = np.concatenate([k for k, _ in merged])
        mv = np.concatenate([v for _, v in merged])
        order = np.argsort(mk)
        assert np.array_equal(mk[order], ok) and np.array_equal(mv[order], ov)
        # Omega_t' from the gathered candidates, then Omega_t.
        allc = torch.cat(cands)
        sel, ns = ops[0].select(allc, allc.shape[0], tprime)
        ref_c, nref = mad.mad_topk(one.ctx.ctx, tprime)
        assert ns == nref
        assert np.array_equal(sel[:ns].cpu().numpy(), ref_c[:nref].cpu().numpy())
        res, nr = ops[0].rescore(sel, ns, t)
        ref, nrr = mad.mad_rescore(one.ctx.ctx, ref_c, nref, t)
        assert nr == nrr
        assert np.array_equal(res[:nr].cpu().numpy(), ref[:nrr].cpu().numpy())
        keys, c = one.oracle.run(s, seed, tprime, t)
        gi, gj, _, gc = mad.decode_pairs(res, nr)
        assert np.array_equal(mad.keys_of(gi, gj), keys)
        assert np.array_equal(gc.view(np.int64), c.view(np.int64))
    finally:
        for c in ranks + [one]:
            c.close()


def test_select_pairs_orders_and_filters():
    """x <= 0 is never selected; ties in x go to the smaller key; fewer
    positive pairs than K returns them all."""
    import paper_1506_03872_gb300 as mad
    c = Case("plain_small", s_max=1 << 16)
    try:
        i = np.array([5, 3, 9, 3, 1, 7])
        j = np.array([1, 2, 0, 1, 4, 7])
        x = np.array([4, 4, -2, 9, 0, 4])
        pairs = mad.encode_pairs(i, j, x)
        out, n = mad.mad_select_pairs(c.ctx.ctx, pairs, 6, 10)
        gi, gj, gx, _ = mad.decode_pairs(out, n)
        assert n == 4
        assert list(zip(gi.tolist(), gj.tolist(), gx.tolist())) == [
            (3, 1, 9), (3, 2, 4), (5, 1, 4), (7, 7, 4)]
        out, n = mad.mad_select_pairs(c.ctx.ctx, pairs, 6, 2)
        assert n == 2
    finally:
        c.close()
