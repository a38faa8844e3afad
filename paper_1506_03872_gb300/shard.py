"""Diamond sampling over several ranks, one GPU each (Alg. 2, then Alg. 3).

Diamonds are independent and indexed by a counter (diamond l draws from the
Philox counter l), so a run of s diamonds splits into contiguous diamond
ranges, one per rank, over tables that every rank builds for itself with
the same budget s (the fixed-point scale depends on it).  X is an exact
integer sum, so summing the ranks' partial X by key gives the X of one run.

The one exchange step routes each partial (key, x) to the key's owner rank
(an all-to-all).  Each owner sums the partials of its keys and selects its
top t' (Alg. 3, first step).  Every key of the global top t' by (x desc, key
asc) is among its owner's top t', so the all-gathered owner candidates hold
the global Omega_t': every rank selects it from them and rescores it (Alg.
3, remaining steps).  The result is bit-identical to one run of s diamonds.

The collectives are torch.distributed's (NCCL between GPUs; the CPU tests
run the same protocol over gloo).  Every compute step is a call of the
library (``LibraryOps``): sampling a diamond range, exporting X grouped by
owner, adding received partials to X, the top-t' selections and the
rescore.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def diamond_range(s: int, rank: int, world: int) -> Tuple[int, int]:
    """(first, count): rank's contiguous share of diamonds [0, s)."""
    first = s * rank // world
    return first, s * (rank + 1) // world - first


def exchange_by_owner(keys, vals, offsets, dist, group=None):
    """All-to-all of the owner segments: segment o of (keys, vals), i.e.
    entries [offsets[o], offsets[o + 1]), goes to rank o.  Returns the
    (keys, vals) this rank received, in sending-rank order."""
    import torch
    send = torch.as_tensor(np.diff(np.asarray(offsets, dtype=np.int64)), dtype=torch.int64,
                           device=keys.device)
    recv = torch.empty_like(send)
    dist.all_to_all_single(recv, send, group=group)
    in_splits, out_splits = send.tolist(), recv.tolist()
    rk = torch.empty(int(sum(out_splits)), dtype=torch.int64, device=keys.device)
    rv = torch.empty_like(rk)
    dist.all_to_all_single(rk, keys.contiguous(), out_splits, in_splits, group=group)
    dist.all_to_all_single(rv, vals.contiguous(), out_splits, in_splits, group=group)
    return rk, rv


def all_gather_pairs(pairs, n: int, dist, group=None):
    """Every rank's first n pair records (n may differ between ranks),
    concatenated in rank order: (pairs, total)."""
    import torch
    world = dist.get_world_size(group)
    cnt = torch.tensor([n], dtype=torch.int64, device=pairs.device)
    counts = [torch.empty_like(cnt) for _ in range(world)]
    dist.all_gather(counts, cnt, group=group)
    counts = [int(c.item()) for c in counts]
    width = max(1, max(counts))
    mine = torch.zeros((width, 3), dtype=torch.int64, device=pairs.device)
    mine[:n] = pairs[:n]
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    out = torch.cat([p[:c] for p, c in zip(parts, counts)]) if sum(counts) else mine[:0]
    return out, int(sum(counts))


class LibraryOps:
    """The compute steps of a sharded run as library calls on this rank's
    GPU (context ``ctx``, tables built with the full budget s)."""

    def __init__(self, ctx, export_cap: int = 1 << 20):
        self.ctx = ctx
        self.cap = export_cap

    def sample(self, count: int, seed: int, first: int) -> None:
        import paper_1506_03872_gb300 as mad
        mad.mad_sample(self.ctx, count, seed, first)

    def export_by_owner(self, world: int):
        import paper_1506_03872_gb300 as mad
        keys, vals, offsets = mad.mad_export_x_by_owner(self.ctx, world, self.cap)
        self.cap = max(self.cap, int(offsets[-1]))
        return keys, vals, offsets

    def reset(self) -> None:
        import paper_1506_03872_gb300 as mad
        mad.mad_reset_hash(self.ctx)

    def accumulate(self, keys, vals) -> None:
        import paper_1506_03872_gb300 as mad
        mad.mad_accumulate(self.ctx, keys, vals)

    def topk(self, tprime: int):
        import paper_1506_03872_gb300 as mad
        return mad.mad_topk(self.ctx, tprime)

    def select(self, pairs, n: int, K: int):
        import paper_1506_03872_gb300 as mad
        return mad.mad_select_pairs(self.ctx, pairs, n, K)

    def rescore(self, pairs, n: int, t: int):
        import paper_1506_03872_gb300 as mad
        return mad.mad_rescore(self.ctx, pairs, n, t)


def sharded_run(ops, dist, s: int, seed: int, tprime: int, t: int, group=None):
    """One sharded pass of s diamonds (Alg. 2 then Alg. 3) on this rank:
    returns (Omega_t pairs, count), the same on every rank and the same as
    one run of s diamonds."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    first, count = diamond_range(s, rank, world)
    ops.sample(count, seed, first)                       # partial X of this range
    keys, vals, offsets = ops.export_by_owner(world)     # grouped by owner rank
    rk, rv = exchange_by_owner(keys, vals, offsets, dist, group)
    ops.reset()
    ops.accumulate(rk, rv)                               # X of the keys this rank owns
    cand, nc = ops.topk(tprime)                          # the owner's top t'
    allc, na = all_gather_pairs(cand, nc, dist, group)   # every owner's candidates
    sel, ns = ops.select(allc, na, tprime)               # global Omega_t'
    return ops.rescore(sel, ns, t)                       # Omega_t
