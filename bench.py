"""Benchmark of diamond sampling (arXiv:1506.03872) on GB300.

One step = the whole hot path on one synthetic batch, inputs resident in
HBM: mad_build_tables (weights and cumulative tables), mad_sample (s
diamonds), mad_topk (Omega_t') and mad_rescore (Omega_t).  Default workload:
dense recommender factors, A 200000x100 and B 100x50000 FP32, s = 1e7,
t = 100, t' = 1e4.

Prints one JSON line.  value = diamonds per second over whole steps
(device-timed, CUDA events, L2 flushed between steps); e2e = the same metric
through the C ABI with the inputs copied from pinned host memory and the
top-t read back inside the timed region.

--impl reference times the CPU oracle on a bounded sample of the same
workload (the reference arm of this comparison).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1506_03872_gb300.truth import (ground_truth_dense, ground_truth_gram_binary,  # noqa: E402
                                            mad_keys, recall_of)

METRIC = "time-to-top-t at recall>=0.95 vs dense GEMM+top-t on 1 GB300; diamonds/sec"
SAMPLER_SOURCES = ["paper_1506_03872_gb300/csrc/sample.cu",
                   "paper_1506_03872_gb300/csrc/draw.cuh",
                   "paper_1506_03872_gb300/csrc/mad_device.cuh"]
# Algorithmic bytes per diamond of the dominant kernel, one 32-byte sector
# per random touch.  Dense draw kernel (k_sample_sorted): the final entry of
# each of the four inverse-CDF searches (T1, T2, TA, TB) and b_k'j, plus the
# 4-byte diamond index read in row order and the 16-byte (key, increment)
# record written.
DENSE_DRAW_BYTES = 32 * 5 + 4 + 16
# 0/1 draw kernel (k_sample, draws and inserts): the final entry of the T1
# search, row i's bounds, the T2 guide entries and the T2 window, the column
# indices of k and k', row k's bounds, b_kj's index and the closure filter's
# word (the exact closure search of the ~1 % of diamonds the filter passes
# is left out); the hash read-modify-write of closed diamonds is added per
# inserted diamond (2 sectors read and written).
SPARSE_DRAW_SECTORS = 9
HASH_RMW_BYTES = 4 * 32
DENSE_DRAW_SECTORS = 5
# Region builder (k_group_prep + k_build_x) of the fused pass: each diamond's
# 16-byte (key, increment) record read once, each slot of the home regions
# (16 bytes) written once.
BUILD_RECORD_BYTES = 16
SLOT_BYTES = 16


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _bf16_peak():
    """Dense BF16 tensor peak (TFLOP/s) of a kernel timed alone: the
    measured cuBLAS burst figure, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def dense_table_bytes(w):
    """Bytes of the tables a dense diamond's draws read at random: T2 and TA
    (m x d uint32), TB (d x n uint32), B (d x n FP32) and T1 (m uint64)."""
    return 8 * w.m * w.d + 8 * w.d * w.n + 8 * w.m


def sparse_table_bytes(w):
    """Bytes of the tables a 0/1 diamond's draws read at random: T1 and the
    row pointers (8 bytes per row each), T2 and the column indices (4 bytes
    per stored entry each)."""
    nnz = int(w.rowptr[-1])
    return 16 * w.m + 8 * nnz


def run_probes(mad, dev, stream, gather_bytes, atomic_bytes=None, count=1 << 26, reps=3):
    """The random-access ceilings: 4-byte loads from random 32-byte sectors
    of a buffer of `gather_bytes`, and random 64-bit atomics (add and
    compare-and-swap) on a buffer of `atomic_bytes` (median of `reps` event-
    timed launches after one warm-up)."""
    import torch
    out = {}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    sink = torch.zeros(4, dtype=torch.int64, device=dev)
    gb = (int(gather_bytes) + 31) // 32 * 32
    table = torch.ones(gb // 4, dtype=torch.int32, device=dev)
    ms = timed(lambda: mad.mad_probe_gather(table, count, 7, sink))
    out["gather"] = {"table_bytes": gb, "loads": count, "ms": round(ms, 4),
                     "sectors_per_s": round(count / (ms / 1e3), 1),
                     "gbs_32b_sectors": round(32 * count / (ms / 1e3) / 1e9, 1)}
    del table
    if atomic_bytes:
        ab = (int(atomic_bytes) + 7) // 8 * 8
        words = torch.zeros(ab // 8, dtype=torch.int64, device=dev)
        for mode, name in ((0, "atomic_add"), (1, "atomic_cas")):
            ms = timed(lambda: mad.mad_probe_atomics(words, count, mode, 11, sink))
            out[name] = {"table_bytes": ab, "ops": count, "ms": round(ms, 4),
                         "ops_per_s": round(count / (ms / 1e3), 1)}
        del words
    torch.cuda.synchronize()
    return out


def _roof(kernel, alg_bytes, kernel_ms, peak, peak_kind, diamonds, sectors=None, probe=None):
    """Roofline entry: algorithmic bytes per launch over the event-timed
    duration, against the measured copy bandwidth; for gather-bound kernels
    also its random sectors per second against the probe's rate."""
    achieved = alg_bytes / (kernel_ms / 1e3) / 1e9
    rec = _traffic_record(kernel)
    traffic = round(rec["bytes_per_diamond"] * diamonds) if rec else None
    r = {"bound": "hbm", "kernel": kernel, "achieved": round(achieved, 1), "peak": peak,
         "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
         "traffic": traffic, "algorithmic_bytes_per_launch": int(alg_bytes),
         "kernel_ms": round(kernel_ms, 4)}
    if traffic is not None:
        dram_gbs = traffic / (kernel_ms / 1e3) / 1e9
        r["dram_gbs"] = round(dram_gbs, 1)
        r["dram_frac"] = round(dram_gbs / peak, 4)
    if sectors is not None and probe:
        rate = sectors / (kernel_ms / 1e3)
        r["random_sectors_per_s"] = round(rate, 1)
        r["gather_probe_sectors_per_s"] = probe["sectors_per_s"]
        r["frac_of_gather_probe"] = round(rate / probe["sectors_per_s"], 4)
    return r


def _sources_sha():
    h = hashlib.sha256()
    for p in SAMPLER_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_record(kernel):
    """DRAM bytes per diamond of `kernel` from an ncu capture, valid only
    while the sampler sources are the ones it was taken with."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec.get("source_sha") == _sources_sha() and kernel in rec.get("kernels", {}):
            return rec["kernels"][kernel]
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons (background)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def start(self):
        self._stop.clear()

        def run():
            while not self._stop.is_set():
                try:
                    out = subprocess.run(
                        ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                         "--format=csv,noheader,nounits"], capture_output=True, text=True,
                        timeout=5).stdout.strip()
                    if out:
                        self.rows.append([x.strip() for x in out.split(",")])
                except Exception:
                    pass
                self._stop.wait(0.2)
        self._t = threading.Thread(target=run, daemon=True)
        self._t.start()

    def stop(self):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in self.rows for q in range(4)
                          if len(r) > 4 + q and r[4 + q].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch.distributed as dist
    dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND") != "gloo" else "gloo")
    return dist, dist.get_rank(), ws


def max_over_ranks(dist, value: float, device=None) -> float:
    """Largest value over all ranks (the slowest rank sets the job time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _workload(name: str, scale: float):
    from paper_1506_03872_gb300 import workloads as W
    if name == "dense_factors":
        if scale != 1.0:
            return W.dense_factors(m=int(200_000 * scale), n=int(50_000 * scale),
                                   s=int(10_000_000 * scale))
        return W.dense_factors()
    if name == "plain_small":
        return W.plain_small()
    if name == "chung_lu":
        return W.chung_lu()
    raise KeyError(name)






def _ladder(step, w, truth, tau, counts, flush, s_max_bytes, seeds, stream, recall_at_s):
    """Time to top-t at recall >= 0.95: the smallest s on {1,2,5} x 10^k
    whose median recall over `seeds` sampler seeds reaches 0.95.  The walk
    starts at the workload's s and goes up while the median falls short, or
    down while it still reaches the target.  Each rung is one warm-up, then
    one timed step per seed (L2 flushed before each)."""
    import torch

    import paper_1506_03872_gb300 as mad
    ladder = [m * 10 ** e for e in range(3, 12) for m in (1, 2, 5)]
    q0 = min(range(len(ladder)), key=lambda q: abs(np.log(ladder[q] / w.s)))
    up = recall_at_s < 0.95
    rungs = []
    result = {"rungs": rungs, "s": None, "ms": None, "recall": None}

    def run(s):
        rec, ms = [], []
        step(s, w.sampler_seed)   # warm-up at this s (sizes the hash)
        for q in range(seeds):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res, nr = step(s, w.sampler_seed + q)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            gi, gj, gx, gc = mad.decode_pairs(res, nr)
            rec.append(recall_of(w, gi, gj, gc, truth, tau, counts)[0])
        r = {"s": s, "recall_median": float(np.median(rec)),
             "ms_median": round(float(np.median(ms)), 3)}
        rungs.append(r)
        return r

    q = q0
    while 0 <= q < len(ladder):
        s = ladder[q]
        if hash_bytes_estimate(w, s) > s_max_bytes:
            result["stopped"] = f"s={s} needs more device memory than the cap"
            break
        r = run(s)
        if r["recall_median"] >= 0.95:
            result.update(s=s, ms=r["ms_median"], recall=r["recall_median"])
            if up:
                break
            q -= 1
        elif not up and result["s"] is None:
            up = True   # one seed reached the target at this s, the median did not
            q += 1
        elif not up:
            break
        else:
            q += 1
    return result


def hash_bytes_estimate(w, s):
    """Device bytes the library allocates for the hash at budget s: 16-byte
    slots, m + 3s of them for dense inputs (per-row regions), else the power
    of two at or above s / 0.6."""
    if w.csr:
        cap = 1024
        while cap < s / 0.6:
            cap <<= 1
        return 16 * cap
    return 16 * (w.m + 3 * s + 1)


def run_ours(args):
    import torch

    import paper_1506_03872_gb300 as mad
    from paper_1506_03872_gb300 import build as _build
    dist, rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    _build.build()
    w = _workload(args.workload, args.scale)
    if getattr(args, "square_sym", False):
        if not w.csr:
            raise SystemExit("--square-sym needs a 0/1 Gram workload")
        w.flags |= 8
    s, t, tprime, seed = w.s, w.t, w.tprime, w.sampler_seed
    dev = torch.device("cuda", local)
    if w.csr:
        tensors = [torch.from_numpy(x).to(dev) for x in (w.rowptr, w.colidx)]
        Am = mad.csr(tensors[0], tensors[1], (w.m, w.d))
        Bm = Am
        host_inputs = [torch.from_numpy(x).pin_memory() for x in (w.rowptr, w.colidx)]
    else:
        tensors = [torch.from_numpy(w.A).to(dev), torch.from_numpy(w.B).to(dev)]
        Am, Bm = mad.dense(tensors[0]), mad.dense(tensors[1])
        host_inputs = [torch.from_numpy(w.A).pin_memory(), torch.from_numpy(w.B).pin_memory()]
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ctx = mad.Context(w.flags)
    out_c = mad.new_pairs(tprime)
    out_t = mad.new_pairs(t)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(A_, B_, timing=None, s_=None, seed_=None):
        s_ = s if s_ is None else s_
        seed_ = seed if seed_ is None else seed_
        e = [ev() for _ in range(5)] if timing is not None else None
        if e: e[0].record(stream)
        mad.mad_build_tables(ctx.ctx, A_, B_, s_)
        if e: e[1].record(stream)
        mad.mad_sample(ctx.ctx, s_, seed_)
        if e: e[2].record(stream)
        cand, nc = mad.mad_topk(ctx.ctx, tprime, out_c)
        if e: e[3].record(stream)
        res, nr = mad.mad_rescore(ctx.ctx, cand, nc, t, out_t)
        if e: e[4].record(stream)
        if timing is not None:
            timing.append(e)
        return res, nr

    for _ in range(args.warmup):
        step(Am, Bm)
    torch.cuda.synchronize()
    launches0 = mad.mad_stats(ctx.ctx)["launches"]
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks: clocks.start()
    if dist: dist.barrier()
    torch.cuda.synchronize()
    timings = []
    phase_events = []
    for _ in range(args.steps):
        flush.fill_(1.0)   # evict the 129 MB L2 between timed steps
        pe = [ev() for _ in range(4)]
        mad.mad_set_phase_events(ctx.ctx, pe)
        phase_events.append(pe)
        step(Am, Bm, timings)
    torch.cuda.synchronize()
    mad.mad_set_phase_events(ctx.ctx, [])
    # sampling phases: row-order sort, draw kernel, hash insert
    phase_kernels = [[pe[q].elapsed_time(pe[q + 1]) for q in range(3)] for pe in phase_events]
    if dist: dist.barrier()
    clk = clocks.stop() if clocks else None
    launches = mad.mad_stats(ctx.ctx)["launches"] - launches0
    phase = np.array([[e[q].elapsed_time(e[q + 1]) for q in range(4)] for e in timings])
    step_ms = phase.sum(axis=1)
    total_ms = max_over_ranks(dist, float(step_ms.sum()), dev)
    ms_per_step = total_ms / args.steps
    value = world * s * args.steps / (total_ms / 1e3)

    # Recall of the last step against exact ground truth (not timed).
    res, nr = step(Am, Bm)
    gi, gj, gx, gc = mad.decode_pairs(res, nr)
    recall = None
    tau = None
    truth = set()
    counts = None
    mismatch = None
    top1 = None
    if rank == 0 and not args.no_recall:
        if w.csr:
            tau, counts = ground_truth_gram_binary(w.rowptr, w.colidx, t, dev)
            top1 = counts.top1
        else:
            truth, tau = ground_truth_dense(tensors[0], tensors[1], t)
            top1 = ground_truth_dense.top1
        recall, mismatch = recall_of(w, gi, gj, gc, truth, tau, counts)
    stats = mad.mad_stats(ctx.ctx)

    # Dense inputs: the fused pass (mad_pipeline_run) captured once in a CUDA
    # graph and replayed, the whole of Alg. 2 and Alg. 3 per replay with no
    # host round trip.  It is the headline step; the step-wise calls above
    # give the phase split and the draw-kernel time.
    pipe = None
    pass_kernels = None
    pass_regions = 0
    step_ms_stepwise = ms_per_step
    if not w.csr:
        mad.mad_pipeline_plan(ctx.ctx, Am, Bm, s, tprime, t)
        p_out, p_cand = mad.new_pairs(t), mad.new_pairs(tprime)
        p_cnt = torch.zeros(2, dtype=torch.int32, device=dev)
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            l0 = mad.mad_stats(ctx.ctx)["launches"]
            mad.mad_pipeline_run(ctx.ctx, seed, p_out, p_cnt, p_cand)
            launches_per_pass = mad.mad_stats(ctx.ctx)["launches"] - l0
        stream.wait_stream(side)
        torch.cuda.synchronize()
        mad.mad_pipeline_status(ctx.ctx)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            mad.mad_pipeline_run(ctx.ctx, seed, p_out, p_cnt, p_cand)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        if clocks: clocks.start()
        if dist: dist.barrier()
        torch.cuda.synchronize()
        pms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            g0, g1 = ev(), ev()
            g0.record(stream)
            graph.replay()
            g1.record(stream)
            pms.append((g0, g1))
        torch.cuda.synchronize()
        if dist: dist.barrier()
        clk = clocks.stop() if clocks else clk
        mad.mad_pipeline_status(ctx.ctx)
        pipe_total = max_over_ranks(dist, float(sum(a.elapsed_time(b_) for a, b_ in pms)), dev)
        nc_p, nr_p = [int(v) for v in p_cnt.cpu().numpy()]
        same = (nr_p == nr and torch.equal(p_out[:nr_p].cpu(), res[:nr].cpu()))
        pipe = {"ms_per_step": round(pipe_total / args.steps, 4), "graph": True,
                "launches_per_pass": int(launches_per_pass),
                "candidates": nc_p, "results": nr_p, "matches_stepwise": bool(same)}
        ms_per_step = pipe_total / args.steps
        value = world * s * args.steps / (pipe_total / 1e3)
        launches = launches_per_pass * args.steps
        # Kernel times inside the fused pass: the same pass enqueued directly
        # (the graph holds the same launches) with the library's events around
        # the row-order sort, the draws and the region builder.
        pk = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            pe = [ev() for _ in range(4)]
            mad.mad_set_phase_events(ctx.ctx, pe)
            mad.mad_pipeline_run(ctx.ctx, seed, p_out, p_cnt, p_cand)
            pk.append(pe)
        torch.cuda.synchronize()
        mad.mad_set_phase_events(ctx.ctx, [])
        mad.mad_pipeline_status(ctx.ctx)
        pass_kernels = {k: float(np.mean([pe[q].elapsed_time(pe[q + 1]) for pe in pk]))
                        for q, k in enumerate(["row_order", "draws", "build_x"])}
        pipe["kernels_ms"] = {k: round(v, 4) for k, v in pass_kernels.items()}
        pass_regions = int(mad.mad_stats(ctx.ctx)["hash_capacity"])

    # End to end from pinned host memory through the C ABI.  Dense inputs:
    # every step copies its 100 MB of inputs from pinned host memory into a
    # plan's input buffers, replays the plan's pass and reads Omega_t back
    # into pinned host memory.  Two plans (contexts with their own input
    # buffers and graphs) alternate, so the copy of step k + 1 runs on a
    # copy stream while step k's pass runs.  0/1 inputs: the step-wise calls
    # on freshly copied inputs.
    e2e_ms = []
    e2e_note = None
    if pipe is not None:
        ctx2 = mad.Context(w.flags)
        tensors2 = [torch.empty_like(x) for x in tensors]
        mad.mad_pipeline_plan(ctx2.ctx, mad.dense(tensors2[0]), mad.dense(tensors2[1]), s,
                              tprime, t)
        p_out2, p_cand2 = mad.new_pairs(t), mad.new_pairs(tprime)
        p_cnt2 = torch.zeros(2, dtype=torch.int32, device=dev)
        for dst, h in zip(tensors2, host_inputs):
            dst.copy_(h)
        side2 = torch.cuda.Stream()
        side2.wait_stream(stream)
        with torch.cuda.stream(side2):
            mad.mad_pipeline_run(ctx2.ctx, seed, p_out2, p_cnt2, p_cand2)
        stream.wait_stream(side2)
        torch.cuda.synchronize()
        graph2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph2):
            mad.mad_pipeline_run(ctx2.ctx, seed, p_out2, p_cnt2, p_cand2)
        plans = [(tensors, graph, p_out, p_cnt), (tensors2, graph2, p_out2, p_cnt2)]
        host_res = [torch.empty(p_out.shape, dtype=p_out.dtype).pin_memory() for _ in range(2)]
        host_cnt = [torch.empty(2, dtype=torch.int32).pin_memory() for _ in range(2)]
        copy_stream = torch.cuda.Stream()
        copied = [torch.cuda.Event() for _ in range(2)]
        used = [torch.cuda.Event() for _ in range(2)]
        for reps, timed in ((args.warmup, False), (args.steps, True)):
            torch.cuda.synchronize()
            a0, a1 = ev(), ev()
            a0.record(stream)
            copy_stream.wait_event(a0)
            for q in range(reps):
                b = q & 1
                bufs, g, outp, cntp = plans[b]
                if q >= 2:
                    copy_stream.wait_event(used[b])   # the pass that read these buffers
                with torch.cuda.stream(copy_stream):
                    for dst, h in zip(bufs, host_inputs):
                        dst.copy_(h, non_blocking=True)
                copied[b].record(copy_stream)
                stream.wait_event(copied[b])
                g.replay()
                used[b].record(stream)
                host_res[b].copy_(outp, non_blocking=True)
                host_cnt[b].copy_(cntp, non_blocking=True)
            a1.record(stream)
            torch.cuda.synchronize()
            if timed:
                e2e_ms.append(a0.elapsed_time(a1))
        e2e_total = max_over_ranks(dist, float(sum(e2e_ms)), dev)
        res_e = host_res[(args.steps - 1) & 1]
        nres_e = int(host_cnt[(args.steps - 1) & 1][1])
        same_e = (nres_e == nr and torch.equal(res_e[:nres_e], res[:nr].cpu()))
        h2d = int(sum(h.numel() * h.element_size() for h in host_inputs))
        d2h = int(host_res[0].numel() * host_res[0].element_size() +
                  host_cnt[0].numel() * host_cnt[0].element_size())
        e2e_note = {"plans": 2, "overlap": "step k+1's input copy runs during step k's pass",
                    "l2": "not flushed: each step copies 100 MB of inputs and its pass touches "
                          "about 0.7 GB", "matches_stepwise": bool(same_e)}
        mad.mad_pipeline_status(ctx.ctx)
        mad.mad_pipeline_status(ctx2.ctx)
        ctx2.close()
    else:
        for q in range(args.warmup + args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            a0, a1 = ev(), ev()
            a0.record(stream)
            dev_inputs = [h.to(dev, non_blocking=True) for h in host_inputs]
            A_ = mad.csr(dev_inputs[0], dev_inputs[1], (w.m, w.d))
            res_e, nr_e = step(A_, A_)
            host_res1 = res_e[:nr_e].cpu()
            a1.record(stream)
            torch.cuda.synchronize()
            if q >= args.warmup:
                e2e_ms.append(a0.elapsed_time(a1))
        e2e_total = max_over_ranks(dist, float(sum(e2e_ms)), dev)
        h2d = int(sum(h.numel() * h.element_size() for h in host_inputs))
        d2h = int(host_res1.numel() * host_res1.element_size())

    # Rooflines of the pass's two largest kernels: algorithmic bytes per
    # launch over the kernel's event-timed duration, against the measured
    # copy bandwidth, with the measured random-sector gather rate of a
    # table of the same size beside the draws (their bound).
    sample_ms = float(phase[:, 1].mean())
    phase_k = np.array(phase_kernels) if phase_kernels else None
    peak, peak_kind = _peaks()
    probes = None
    if not args.no_probes:
        probes = run_probes(mad, dev, stream, gather_bytes=dense_table_bytes(w) if not w.csr
                            else sparse_table_bytes(w),
                            atomic_bytes=(16 * int(stats["hash_capacity"]) if w.csr else None))
    rooflines = {}
    if pass_kernels is not None:
        rooflines["k_sample_sorted"] = _roof(
            "k_sample_sorted", DENSE_DRAW_BYTES * s, pass_kernels["draws"], peak, peak_kind, s,
            sectors=DENSE_DRAW_SECTORS * s, probe=(probes or {}).get("gather"))
        rooflines["k_build_x"] = _roof(
            "k_build_x", BUILD_RECORD_BYTES * s + SLOT_BYTES * pass_regions,
            pass_kernels["build_x"], peak, peak_kind, s)
    elif phase_k is not None:
        draw_ms = float(phase_k[:, 1].mean())
        if w.csr:
            rooflines["k_sample"] = _roof(
                "k_sample", 32 * SPARSE_DRAW_SECTORS * s + HASH_RMW_BYTES * int(stats["inserted"]),
                draw_ms, peak, peak_kind, s, sectors=SPARSE_DRAW_SECTORS * s,
                probe=(probes or {}).get("gather"))
        else:
            rooflines["k_sample_sorted"] = _roof(
                "k_sample_sorted", DENSE_DRAW_BYTES * s, draw_ms, peak, peak_kind, s,
                sectors=DENSE_DRAW_SECTORS * s, probe=(probes or {}).get("gather"))
    roof = max(rooflines.values(), key=lambda r: r["kernel_ms"]) if rooflines else None

    # The dense exact comparator (BF16 tensor-core GEMM + fused top filter +
    # FP32 rescore) on the same inputs, timed the same way.
    comp = None
    if not w.csr and not args.no_comparator:
        try:
            out_cmp = mad.new_pairs(t)
            for _ in range(max(2, args.warmup)):
                mad.mad_dense_topt(ctx.ctx, Am, Bm, t, args.rescore, out=out_cmp)
            cms = []
            for _ in range(args.steps):
                flush.fill_(1.0)
                c0, c1 = ev(), ev()
                c0.record(stream)
                res_c, nrc = mad.mad_dense_topt(ctx.ctx, Am, Bm, t, args.rescore, out=out_cmp)
                c1.record(stream)
                torch.cuda.synchronize()
                cms.append(c0.elapsed_time(c1))
            ci, cj, _, _ = mad.decode_pairs(res_c, nrc)
            k_issued = 16 * ((w.d + 15) // 16)   # the MMAs stop at the first K step past d
            cm = float(np.mean(cms))
            useful = 2.0 * w.m * w.n * w.d / (cm / 1e3) / 1e12
            bpeak, bkind = _bf16_peak()
            comp = {"kernel": "k_gemm_topk", "ms": round(cm, 4),
                    "rescore": args.rescore or 8 * t,
                    "tflops_useful": round(useful, 1),
                    "tflops_issued": round(2.0 * w.m * w.n * k_issued / (cm / 1e3) / 1e12, 1),
                    # The whole call (casts, norm order, threshold pre-pass,
                    # GEMM with its filter, selections, FP32 rescore) against
                    # the bf16 burst peak: useful FLOPs 2 m n d.
                    "roofline": {"bound": "tensor", "achieved": round(useful, 1), "peak": bpeak,
                                 "peak_kind": bkind, "unit": "TFLOP/s",
                                 "frac": round(useful / bpeak, 4)}}
            if recall is not None:
                got_c = set(mad.keys_of(ci, cj).astype(np.int64).tolist())
                comp["recall"] = len(got_c & truth) / t
        except Exception as ex:  # the comparator must not cost the main line
            comp = {"error": str(ex)[:200]}

    # Alias-table draws (MAD_ALIAS, Sec. 4.1) on the same inputs and budget:
    # the same law through another map from the uniforms, diamonds in index
    # order.  Tables, sampling and the whole step, timed like the main line.
    alias_leg = None
    if rank == 0 and not w.csr and not args.no_alias:
        try:
            actx = mad.Context(w.flags | mad.MAD_ALIAS)
            a_out_c, a_out_t = mad.new_pairs(tprime), mad.new_pairs(t)

            def astep():
                e = [ev() for _ in range(4)]
                e[0].record(stream)
                mad.mad_build_tables(actx.ctx, Am, Bm, s)
                e[1].record(stream)
                mad.mad_sample(actx.ctx, s, seed)
                e[2].record(stream)
                cand_a, nc_a = mad.mad_topk(actx.ctx, tprime, a_out_c)
                res_a, nr_a = mad.mad_rescore(actx.ctx, cand_a, nc_a, t, a_out_t)
                e[3].record(stream)
                return e, res_a, nr_a
            for _ in range(max(2, args.warmup)):
                astep()
            aev = []
            for _ in range(args.steps):
                flush.fill_(1.0)
                e, res_a, nr_a = astep()
                aev.append(e)
            torch.cuda.synchronize()
            at = np.array([[e[q].elapsed_time(e[q + 1]) for q in range(3)] for e in aev])
            alias_leg = {"tables_ms": round(float(at[:, 0].mean()), 4),
                         "sample_ms": round(float(at[:, 1].mean()), 4),
                         "step_ms": round(float(at.sum(axis=1).mean()), 4),
                         "diamonds_per_s_sampler": round(s / (float(at[:, 1].mean()) / 1e3), 1),
                         "prefix_table_sample_ms": round(sample_ms, 4)}
            if recall is not None:
                ai, aj, _, ac = mad.decode_pairs(res_a, nr_a)
                alias_leg["recall_at_s"] = recall_of(w, ai, aj, ac, truth, tau, counts)[0]
            actx.close()
        except Exception as ex:  # the alias leg must not cost the main line
            alias_leg = {"error": str(ex)[:200]}

    # 0/1 inputs: the exact sparse comparator (degree-bounded row-block
    # product with a fused threshold) on the same inputs, timed the same way.
    if w.csr and not args.no_comparator:
        try:
            out_x = mad.new_pairs(t)
            for _ in range(2):
                mad.mad_sparse_topt(ctx.ctx, Am, Bm, t, 0, out_x)
            cms = []
            for _ in range(args.steps):
                flush.fill_(1.0)
                c0, c1 = ev(), ev()
                c0.record(stream)
                res_x, nx = mad.mad_sparse_topt(ctx.ctx, Am, Bm, t, 0, out_x)
                c1.record(stream)
                torch.cuda.synchronize()
                cms.append(c0.elapsed_time(c1))
            comp = {"kernel": "k_spgemm_rowblock_topk", "ms": round(float(np.mean(cms)), 4),
                    "results": int(nx)}
            if counts is not None:
                xi, xj, _, xc = mad.decode_pairs(res_x, nx)
                comp["recall"], comp["count_mismatches"] = recall_of(w, xi, xj, xc, set(), tau,
                                                                     counts)
        except Exception as ex:  # the comparator must not cost the main line
            comp = {"error": str(ex)[:200]}

    ladder = None
    if rank == 0 and recall is not None and not args.no_ladder:
        try:
            free, _ = torch.cuda.mem_get_info(dev)
            cap = int(0.6 * free)
            ladder = _ladder(lambda s_, seed_: step(Am, Bm, s_=s_, seed_=seed_), w, truth, tau,
                             counts, flush, cap, args.ladder_seeds, stream, recall)
        except Exception as ex:  # the ladder must not cost the main line
            ladder = {"error": str(ex)[:200]}

    ctx.close()   # frees the ladder's largest hash before the sparse leg
    sparse = None
    if rank == 0 and not w.csr and args.workload == "dense_factors" and args.scale == 1.0 \
            and not args.no_sparse:
        try:
            sparse = chung_lu_leg(args, dev, stream, flush, peak, peak_kind)
        except Exception as ex:  # the sparse leg must not cost the main line
            sparse = {"error": str(ex)[:300]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, args.cpu_diamonds)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "diamonds/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name + ("+square_sym" if w.flags & 8 else ""), "m": w.m,
                       "d": w.d, "n": w.n, "s": s, "t": t,
                       "tprime": tprime, "flags": w.flags, "l2": "flushed between steps",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "pass": pipe,
            "stepwise_ms_per_step": round(step_ms_stepwise, 4),
            "phases_ms": {k: round(float(phase[:, q].mean()), 4)
                          for q, k in enumerate(["build_tables", "sample", "topk", "rescore"])},
            "diamonds_per_s_sampler": round(s / (sample_ms / 1e3), 1),
            "sample_kernels_ms": ({k: round(float(np.mean([pk[q] for pk in phase_kernels])), 4)
                                   for q, k in enumerate(["row_order", "draws", "insert"])}
                                  if phase_kernels else None),
            "recall_at_s": recall, "tau_t": tau, "count_mismatches": mismatch,
            # Theorem 2's sample estimate for the top entry, ||W||_1 / max c^2
            # (the paper's "est. samples" statistic).
            "est_samples_top1": (round(stats["w1"] / top1 ** 2, 1) if top1 else None),
            "stats": {k: stats[k] for k in ("w1", "inserted", "distinct", "positive",
                                              "hash_capacity")},
            "e2e": {"value": round(world * s * args.steps / (e2e_total / 1e3), 1),
                    "unit": "diamonds/s", "ms_per_step": round(e2e_total / args.steps, 4),
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    **({"pipelined": e2e_note} if e2e_note else {})},
            "gpu_launches": int(launches),
            "comparator": comp,
            "alias": alias_leg,
            "time_to_top_t": {"recall_target": 0.95,
                              "sampling_ms_at_s": round(ms_per_step, 4), "sampling_recall_at_s": recall,
                              "ladder": ladder,
                              "comparator_ms": comp.get("ms") if comp else None,
                              "comparator_recall": comp.get("recall") if comp else None},
            "roofline": roof,
            "rooflines": rooflines,
            "probes": probes,
            "chung_lu": sparse,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def chung_lu_leg(args, dev, stream, flush, peak, peak_kind):
    """The sparse common-neighbours workload (Chung-Lu graph, 1e6 nodes, 0/1
    Gram, diagonal excluded, s = 1e8, t = 1000, t' = 1e5): the step-wise
    sampler timed over whole steps, recall against exact ground truth, the
    time-to-recall ladder, the exact sparse comparator timed the same way,
    and the draw kernel against the measured gather and atomic rates."""
    import torch

    import paper_1506_03872_gb300 as mad
    from paper_1506_03872_gb300 import workloads as W
    w = W.chung_lu()
    rp = torch.from_numpy(w.rowptr).to(dev)
    ci = torch.from_numpy(w.colidx).to(dev)
    A = mad.csr(rp, ci, (w.m, w.d))
    ctx = mad.Context(w.flags)
    out_c, out_t = mad.new_pairs(w.tprime), mad.new_pairs(w.t)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(s_, seed_, c=ctx):
        mad.mad_build_tables(c.ctx, A, A, s_)
        mad.mad_sample(c.ctx, s_, seed_)
        cand, nc = mad.mad_topk(c.ctx, w.tprime, out_c)
        return mad.mad_rescore(c.ctx, cand, nc, w.t, out_t)

    for _ in range(args.warmup):
        step(w.s, w.sampler_seed)
    torch.cuda.synchronize()
    spans, pks = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        pe = [ev() for _ in range(4)]
        mad.mad_set_phase_events(ctx.ctx, pe)
        e0, e1 = ev(), ev()
        e0.record(stream)
        res, nr = step(w.s, w.sampler_seed)
        e1.record(stream)
        spans.append((e0, e1))
        pks.append(pe)
    torch.cuda.synchronize()
    mad.mad_set_phase_events(ctx.ctx, [])
    step_ms = float(np.mean([a.elapsed_time(b) for a, b in spans]))
    draw_ms = float(np.mean([pe[1].elapsed_time(pe[2]) for pe in pks]))
    st = mad.mad_stats(ctx.ctx)
    tau, counts = ground_truth_gram_binary(w.rowptr, w.colidx, w.t, dev)
    gi, gj, gx, gc = mad.decode_pairs(res, nr)
    recall, mismatch = recall_of(w, gi, gj, gc, set(), tau, counts)
    leg = {"workload": w.name, "m": w.m, "nnz": int(w.rowptr[-1]), "s": w.s, "t": w.t,
           "tprime": w.tprime, "flags": w.flags, "ms_per_step": round(step_ms, 4),
           "diamonds_per_s": round(w.s / (step_ms / 1e3), 1), "recall_at_s": recall,
           "count_mismatches": mismatch, "tau_t": tau,
           "est_samples_top1": round(st["w1"] / counts.top1 ** 2, 1) if counts.top1 else None,
           "stats": {k: st[k] for k in ("w1", "inserted", "distinct", "hash_capacity")}}
    # The same step as the fused pass (mad_pipeline_*), planned once and
    # replayed from a CUDA graph: no host round trip inside a step.
    try:
        pctx = mad.Context(w.flags)
        mad.mad_pipeline_plan(pctx.ctx, A, A, w.s, w.tprime, w.t)
        p_out, p_cand = mad.new_pairs(w.t), mad.new_pairs(w.tprime)
        p_cnt = torch.zeros(2, dtype=torch.int32, device=dev)
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            mad.mad_pipeline_run(pctx.ctx, w.sampler_seed, p_out, p_cnt, p_cand)
        stream.wait_stream(side)
        torch.cuda.synchronize()
        mad.mad_pipeline_status(pctx.ctx)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            mad.mad_pipeline_run(pctx.ctx, w.sampler_seed, p_out, p_cnt, p_cand)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        gspans = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            g0, g1 = ev(), ev()
            g0.record(stream)
            graph.replay()
            g1.record(stream)
            gspans.append((g0, g1))
        torch.cuda.synchronize()
        mad.mad_pipeline_status(pctx.ctx)
        nr_p = int(p_cnt[1].item())
        pass_ms = float(np.mean([a.elapsed_time(b) for a, b in gspans]))
        leg["pass"] = {"graph": True, "ms_per_step": round(pass_ms, 4),
                       "diamonds_per_s": round(w.s / (pass_ms / 1e3), 1),
                       "matches_stepwise": bool(nr_p == nr and
                                                torch.equal(p_out[:nr_p].cpu(), res[:nr].cpu()))}
        del graph
        pctx.close()
    except Exception as ex:  # the fused pass must not cost the leg
        leg["pass"] = {"error": str(ex)[:200]}
    cap = int(0.6 * torch.cuda.mem_get_info(dev)[0])
    leg["ladder"] = _ladder(step, w, set(), tau, counts, flush, cap, args.ladder_seeds, stream,
                            recall)
    # Squared symmetric update (Sec. 3.2.3) on the same graph.
    ctx_sq = mad.Context(w.flags | 8)
    leg["ladder_square_sym"] = _ladder(lambda s_, seed_: step(s_, seed_, ctx_sq), w, set(), tau,
                                       counts, flush, cap, args.ladder_seeds, stream, 1.0)
    ctx_sq.close()

    # Wedge sampling (the paper's comparison, Sec. 6.3) on the same graph:
    # its own time to recall 0.95, up to the memory cap.
    ctx_w = mad.Context(w.flags | 16)
    leg["ladder_wedge"] = _ladder(lambda s_, seed_: step(s_, seed_, ctx_w), w, set(), tau,
                                  counts, flush, cap, args.ladder_seeds, stream, 0.0)
    ctx_w.close()

    # Exact sparse comparator (degree-bounded row-block product).
    comp = {}
    out_x = mad.new_pairs(w.t)
    for _ in range(2):
        mad.mad_sparse_topt(ctx.ctx, A, A, w.t, 0, out_x)
    cms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        c0, c1 = ev(), ev()
        c0.record(stream)
        res_x, nx = mad.mad_sparse_topt(ctx.ctx, A, A, w.t, 0, out_x)
        c1.record(stream)
        torch.cuda.synchronize()
        cms.append(c0.elapsed_time(c1))
    xi, xj, _, xc = mad.decode_pairs(res_x, nx)
    r_x, mis_x = recall_of(w, xi, xj, xc, set(), tau, counts)
    comp = {"kernel": "k_spgemm_rowblock_topk", "ms": round(float(np.mean(cms)), 4),
            "recall": r_x, "count_mismatches": mis_x, "results": int(nx),
            "top_count": float(xc[0]) if nx else None,
            "tth_count": float(xc[-1]) if nx else None}
    leg["comparator"] = comp
    lad = leg["ladder"]
    leg["time_to_top_t"] = {"recall_target": 0.95, "sampling_ms": lad.get("ms"),
                            "sampling_s": lad.get("s"), "sampling_recall": lad.get("recall"),
                            "sampling_square_sym_ms": leg["ladder_square_sym"].get("ms"),
                            "wedge_ms": leg["ladder_wedge"].get("ms"),
                            "wedge_s": leg["ladder_wedge"].get("s"),
                            "comparator_ms": comp["ms"], "comparator_recall": r_x}
    if not args.no_probes:
        probes = run_probes(mad, dev, stream, gather_bytes=sparse_table_bytes(w),
                            atomic_bytes=16 * int(st["hash_capacity"]))
        leg["probes"] = probes
        r = _roof("k_sample", 32 * SPARSE_DRAW_SECTORS * w.s + HASH_RMW_BYTES * int(st["inserted"]),
                  draw_ms, peak, peak_kind, w.s, sectors=SPARSE_DRAW_SECTORS * w.s,
                  probe=probes.get("gather"))
        ins_rate = int(st["inserted"]) / (draw_ms / 1e3)
        r["inserts_per_s"] = round(ins_rate, 1)
        r["atomic_cas_probe_ops_per_s"] = probes["atomic_cas"]["ops_per_s"]
        leg["roofline"] = r
    ctx.close()
    return leg


def _ground_truth_rows(Q, B, t):
    """Exact top t of |q . b_j| for every query row (harness only): FP32
    cuBLAS in item blocks with a margin for its rounding, FP64 rescoring of
    the survivors.  Returns one set of item indices per query."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    nq, d = Q.shape
    n = B.shape[1]
    err = 2.0 * d * 2.0 ** -24 * Q.double().norm(dim=1).max().item() * B.double().norm(dim=0).max().item()
    block = 131072
    best_v, best_i = None, None
    for j0 in range(0, n, block):
        c = (Q @ B[:, j0:j0 + block]).abs_()
        v, i = torch.topk(c, min(4 * t, c.shape[1]), dim=1)
        i += j0
        if best_v is None:
            best_v, best_i = v, i
        else:
            best_v, best_i = torch.cat([best_v, v], 1), torch.cat([best_i, i], 1)
            keep = torch.topk(best_v, min(4 * t, best_v.shape[1]), dim=1)
            best_v, best_i = keep.values, torch.gather(best_i, 1, keep.indices)
    theta = best_v[:, t - 1:t] - 2 * err
    truth = []
    Qd, Bd = Q.double(), B.double()
    for q in range(nq):
        cand = best_i[q][best_v[q] >= theta[q]]
        exact = (Qd[q:q + 1] @ Bd[:, cand]).abs().flatten()
        order = torch.argsort(-exact, stable=True)[:t]
        truth.append(set(cand[order].cpu().tolist()))
    return truth


def run_budget(args):
    """The learned-budget experiment (mixed dense/0-1 instances, a perceptron
    trained on their recall curves, evaluated on held-out instances against
    the fixed budget)."""
    from paper_1506_03872_gb300 import budget
    from paper_1506_03872_gb300 import build as _build
    _build.build()
    res = budget.experiment(count=args.budget_instances,
                            log=lambda m: print(m, file=sys.stderr, flush=True))
    line = {"metric": "learned budget: recall achieved and time saved vs the fixed budget",
            "value": res["time_saved_fraction"], "unit": "fraction of fixed-budget time saved",
            "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "learned_budget", "target_recall": budget.TARGET,
                       "fixed_budget": budget.LADDER[-1], "ladder": budget.LADDER},
            **res}
    print(json.dumps(line), flush=True)


def run_batched_queries(args):
    """Batched queries: the launch shape picked by the autotuner
    (paper_1506_03872_gb300/autotune.py), then one graph-captured batch per
    step under the library's default shape and under the tuned one."""
    import torch

    import paper_1506_03872_gb300 as mad
    from paper_1506_03872_gb300 import autotune
    from paper_1506_03872_gb300 import build as _build
    _build.build()
    from paper_1506_03872_gb300.workloads import batched_queries
    kw = {}
    if args.scale != 1.0:
        kw = dict(n=int(1_000_000 * args.scale), nq=int(10_000 * args.scale))
    w = batched_queries(**kw)
    s_q = w.meta["s_per_query"]
    dev = torch.device("cuda", 0)
    tQ, tB = torch.from_numpy(w.A).to(dev), torch.from_numpy(w.B).to(dev)
    ctx = mad.Context()
    t0 = time.perf_counter()
    mad.mad_mips_items(ctx.ctx, mad.dense(tB), w.meta["s_max"])
    items_s = time.perf_counter() - t0
    tuned = autotune.tune_mips(ctx.ctx, tQ, w.d, w.n, s_q, w.tprime, w.t, w.sampler_seed,
                               use_cache=not args.retune,
                               log=lambda m: print(m, file=sys.stderr, flush=True))
    out = mad.new_pairs(w.m * w.t)
    nout = torch.zeros(w.m, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def timed_graph(cfg):
        mad.mad_mips_config(ctx.ctx, **cfg)
        mad.mad_mips_plan(ctx.ctx, s_q, w.tprime, w.t)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(args.warmup):
                mad.mad_mips_run(ctx.ctx, mad.dense(tQ), w.sampler_seed, out, nout)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            mad.mad_mips_run(ctx.ctx, mad.dense(tQ), w.sampler_seed, out, nout)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps, out.cpu().numpy().copy()

    clocks = ClockSampler(0)
    clocks.start()
    ms_default, res_default = timed_graph(autotune.DEFAULT)
    ms, res_tuned = timed_graph(tuned["best"])
    clk = clocks.stop()
    diamonds = int(s_q.sum())
    st = mad.mad_stats(ctx.ctx)
    recall = None
    if not args.no_recall:
        truth = _ground_truth_rows(tQ, tB, w.t)
        res = out.cpu().numpy()
        cnt = nout.cpu().numpy()
        hits = 0
        for q in range(w.m):
            got = set(((res[q * w.t:q * w.t + int(cnt[q]), 0] >> 32) & 0xFFFFFFFF).tolist())
            hits += len(got & truth[q])
        recall = hits / (w.m * w.t)
    line = {
        "metric": METRIC, "value": round(diamonds / (ms / 1e3), 1), "unit": "diamonds/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "items": w.n, "d": w.d, "queries": w.m,
                   "s_per_query": [int(s_q.min()), int(s_q.max())], "diamonds": diamonds,
                   "t": w.t, "tprime": w.tprime, "graph": "one CUDA graph replay per step",
                   "l2": "inputs and hash regions above L2"},
        "queries_per_s": round(w.m / (ms / 1e3), 1),
        "default_shape": {"ms_per_step": round(ms_default, 3),
                          "queries_per_s": round(w.m / (ms_default / 1e3), 1)},
        "tuned_shape": {"shape": tuned["best"], "cached": tuned["cached"],
                        "trials": len(tuned["trials"]),
                        "results_equal_default": bool(np.array_equal(res_tuned, res_default))},
        "recall_top_t": recall,
        "item_tables_s": round(items_s, 3),
        # per replay: the query-row tables, the sampler, the per-query select
        "gpu_launches": 3 * args.steps,
        "device_error": st["device_error"],
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def _oracle_for(w):
    import oracle
    if w.csr:
        M = oracle.Matrix(rowptr=w.rowptr, colidx=w.colidx, shape=(w.m, w.d))
        return oracle.Oracle(M, M, w.flags, w.s)
    return oracle.Oracle(oracle.Matrix(w.A), oracle.Matrix(w.B), w.flags, w.s)


def cpu_model() -> str:
    """The host CPU's model name (lscpu), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


class OraclePool:
    """One oracle per host thread on the same workload.  A run of diamonds
    [0, s) is split into contiguous ranges, one per thread, sampled
    concurrently (the oracle's calls release the interpreter lock); the
    integer maps are merged by key, so the result is the one-thread X."""

    def __init__(self, w, threads):
        import concurrent.futures as cf
        self.w = w
        self.threads = threads
        self.ex = cf.ThreadPoolExecutor(threads)
        t0 = time.perf_counter()
        self.orcs = list(self.ex.map(lambda _: _oracle_for(w), range(threads)))
        self.tables_s = time.perf_counter() - t0

    def sample(self, s):
        bounds = [s * q // self.threads for q in range(self.threads + 1)]
        for o in self.orcs:
            o.reset()
        t0 = time.perf_counter()
        st = list(self.ex.map(lambda q: self.orcs[q].sample(bounds[q + 1] - bounds[q],
                                                            self.w.sampler_seed, bounds[q]),
                              range(self.threads)))
        sec = time.perf_counter() - t0
        if any(st):
            raise RuntimeError(f"oracle sampling failed: {st}")
        return sec

    def merged_x(self):
        parts = [o.x() for o in self.orcs]
        keys = np.concatenate([k for k, _ in parts])
        vals = np.concatenate([v for _, v in parts])
        uk, inv = np.unique(keys, return_inverse=True)
        out = np.zeros(len(uk), np.int64)
        np.add.at(out, inv, vals)
        return uk, out

    def close(self):
        self.ex.shutdown()
        self.orcs = []


def _all_core_diamonds(w, threads):
    """The all-cores leg samples the workload's s, bounded to 1e6 diamonds
    per thread (a few seconds of work per thread)."""
    return int(min(w.s, 1_000_000 * threads))


def cpu_baseline(w, diamonds, threads=None):
    """The oracle on the host cores.  One core: the tables (oracle
    construction), `diamonds` iterations of the sampling loop, top-t' and
    the rescore, each timed.  All cores: one oracle per thread sampling the
    workload's diamonds in contiguous ranges (the X they merge to is checked
    against the one-core X on the common range).  value = the all-cores
    sampling rate (diamonds/s of the Alg. 2 loop, tables excluded)."""
    import oracle
    threads = threads or os.cpu_count() or 1
    diamonds = min(diamonds, w.s)
    t0 = time.perf_counter()
    o = _oracle_for(w)
    tables_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    if o.sample(diamonds, w.sampler_seed):
        raise RuntimeError("oracle sampling failed")
    sample_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    keys, _ = o.topk(w.tprime)
    oracle.topt(keys, o.rescore(keys), w.t)
    post_s = time.perf_counter() - t0
    one_x = o.x()
    del o
    pool = OraclePool(w, threads)
    try:
        check = pool.sample(diamonds)
        mk, mv = pool.merged_x()
        ok = bool(np.array_equal(mk, one_x[0]) and np.array_equal(mv, one_x[1]))
        big = _all_core_diamonds(w, threads)
        par_s = pool.sample(big)
    finally:
        tables_par_s = pool.tables_s
        pool.close()
    return {"value": round(big / par_s, 1), "unit": "diamonds/s", "cores": threads,
            "kind": "oracle", "cpu_model": cpu_model(),
            "sample": (f"all cores: {big} of the {w.s} diamonds of {w.name} in {threads} "
                       f"contiguous ranges, one oracle per thread (Alg. 2 loop only); one core: "
                       f"tables, {diamonds} diamonds, top-t' and rescore timed apart"),
            "all_cores": {"threads": threads, "diamonds": big, "sampling_s": round(par_s, 3),
                          "diamonds_per_s": round(big / par_s, 1),
                          "tables_s_parallel": round(tables_par_s, 3),
                          "merged_x_equals_one_core": ok, "check_s": round(check, 3)},
            "one_core": {"tables_s": round(tables_s, 3), "diamonds": diamonds,
                         "sampling_s": round(sample_s, 3),
                         "diamonds_per_s": round(diamonds / sample_s, 1),
                         "topk_rescore_s": round(post_s, 3)}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = _workload(args.workload, args.scale)
    threads = os.cpu_count() or 1
    diamonds = _all_core_diamonds(w, threads)
    pool = OraclePool(w, threads)
    try:
        for _ in range(args.warmup):
            pool.sample(diamonds)
        secs = [pool.sample(diamonds) for _ in range(args.steps)]
    finally:
        tables_s = pool.tables_s
        pool.close()
    total = sum(secs)
    value = diamonds * args.steps / total
    sample = (f"{diamonds} of the {w.s} diamonds of {w.name} per step (Alg. 2 loop), split in "
              f"{threads} contiguous ranges, one oracle per host thread; tables built once "
              f"({tables_s:.2f} s, not timed per step)")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "diamonds/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "d": w.d, "n": w.n, "s": w.s, "t": w.t,
                   "tprime": w.tprime, "flags": w.flags, "l2": "flushed between steps",
                   "parallelism": "single"},
        "cpu_baseline": {"value": round(value, 1), "unit": "diamonds/s", "cores": threads,
                         "kind": "oracle", "sample": sample, "cpu_model": cpu_model()},
        "e2e": {"value": round(value, 1), "unit": "diamonds/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dense_factors")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--cpu-diamonds", type=int, default=2_000_000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-recall", action="store_true")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--no-ladder", action="store_true",
                    help="skip the time-to-recall ladder over s")
    ap.add_argument("--ladder-seeds", type=int, default=5)
    ap.add_argument("--budget-instances", type=int, default=512)
    ap.add_argument("--square-sym", action="store_true",
                    help="0/1 Gram workloads: the squared-symmetric update of Sec. 3.2.3")
    ap.add_argument("--no-probes", action="store_true", help="skip the gather/atomic probes")
    ap.add_argument("--retune", action="store_true",
                    help="batched queries: search the launch shape again (ignore the cache)")
    ap.add_argument("--no-alias", action="store_true", help="skip the alias-table leg")
    ap.add_argument("--no-sparse", action="store_true",
                    help="skip the sparse common-neighbours leg of the default run")
    ap.add_argument("--rescore", type=int, default=0,
                    help="comparator FP32 rescore budget (0: 8t)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched_queries":
        run_batched_queries(args)
    elif args.workload == "learned_budget":
        run_budget(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
