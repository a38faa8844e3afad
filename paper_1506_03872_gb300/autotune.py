"""Autotuner of the batched-query launch shape (mad_mips_config).

A batch of queries (Alg. 2 and Alg. 3 per query, mad_mips_run) has four
launch parameters that change its speed and none of its results: the size
of each query's hash region (2^region_lg times its budget, rounded up to a
power of two), the diamonds per chunk (256 x chunk_mult), the sampler's
blocks per SM and the threads of each query's selection.  The tuner times
the batch under each choice with CUDA events (a warm-up run, then the
median of ``reps`` runs), walks the parameters one at a time from the
library's defaults (coordinate descent, two sweeps), and keeps the fastest
shape per device, item matrix shape and batch summary in a JSON cache
(``$MAD_TUNE_CACHE``, default ``~/.cache/mad_gb300/mips_tuned.json``).
"""
from __future__ import annotations

import json
import os
from typing import Callable, Dict, Optional

import numpy as np

SPACE = {
    "region_lg": (1, 2),
    "chunk_mult": (1, 2, 4),
    "blocks_per_sm": (0, 2, 3),
    "select_threads": (128, 256, 512),
}
DEFAULT = {"region_lg": 1, "chunk_mult": 1, "blocks_per_sm": 0, "select_threads": 256}


def cache_path() -> str:
    return os.environ.get("MAD_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mad_gb300",
                                       "mips_tuned.json"))


def shape_key(d: int, n: int, s_q, tprime: int, t: int) -> str:
    """Device, item matrix shape and a summary of the batch (query count,
    budget range and total rounded to two significant digits)."""
    import torch
    s = np.asarray(s_q, dtype=np.float64)
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return (f"{dev}|d={d}|n={n}|nq={len(s)}|s=[{int(s.min())},{int(s.max())}]"
            f"|sum={float(f'{s.sum():.2g}')}|tp={tprime}|t={t}")


def load(key: str) -> Optional[Dict]:
    try:
        with open(cache_path()) as f:
            return json.load(f).get(key)
    except (OSError, ValueError):
        return None


def store(key: str, entry: Dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data[key] = entry
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1)
    os.replace(tmp, path)


def time_batch(ctx, Q, s_q, tprime: int, t: int, seed: int, cfg: Dict, out, nout,
               reps: int = 3) -> float:
    """Median event time (ms) of one batch under launch shape cfg."""
    import torch

    import paper_1506_03872_gb300 as mad
    mad.mad_mips_config(ctx, **cfg)
    mad.mad_mips_plan(ctx, s_q, tprime, t)
    Qm = mad.dense(Q)
    mad.mad_mips_run(ctx, Qm, seed, out, nout)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mad.mad_mips_run(ctx, Qm, seed, out, nout)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def tune_mips(ctx, Q, d: int, n: int, s_q, tprime: int, t: int, seed: int, reps: int = 3,
              use_cache: bool = True, log: Callable[[str], None] = lambda m: None) -> Dict:
    """The fastest launch shape of this batch (coordinate descent from the
    defaults over SPACE); returns {"best", "ms", "default_ms", "trials"} and
    caches it.  Leaves the context planned with the best shape."""
    import paper_1506_03872_gb300 as mad
    key = shape_key(d, n, s_q, tprime, t)
    out = mad.new_pairs(len(s_q) * t)
    import torch
    nout = torch.zeros(len(s_q), dtype=torch.int32, device="cuda")
    if use_cache:
        hit = load(key)
        if hit:
            mad.mad_mips_config(ctx, **hit["best"])
            mad.mad_mips_plan(ctx, s_q, tprime, t)
            return dict(hit, cached=True)
    trials = {}

    def measure(cfg):
        k = json.dumps(cfg, sort_keys=True)
        if k not in trials:
            trials[k] = time_batch(ctx, Q, s_q, tprime, t, seed, cfg, out, nout, reps)
            log(f"mips shape {cfg}: {trials[k]:.3f} ms")
        return trials[k]

    best = dict(DEFAULT)
    best_ms = measure(best)
    default_ms = best_ms
    for _ in range(2):
        changed = False
        for name, values in SPACE.items():
            for v in values:
                if v == best[name]:
                    continue
                cfg = dict(best, **{name: v})
                ms = measure(cfg)
                if ms < best_ms:
                    best, best_ms, changed = cfg, ms, True
        if not changed:
            break
    entry = {"best": best, "ms": round(best_ms, 4), "default_ms": round(default_ms, 4),
             "trials": [dict(json.loads(k), ms=round(v, 4)) for k, v in trials.items()]}
    store(key, entry)
    mad.mad_mips_config(ctx, **best)
    mad.mad_mips_plan(ctx, s_q, tprime, t)
    return dict(entry, cached=False)
