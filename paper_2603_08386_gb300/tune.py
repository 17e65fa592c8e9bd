"""Autotuner of the batched detection call.

Times ``ddhf_detect_batch`` on the caller's own windows for each candidate
``ddhf_tuning`` (heavy-pixel threshold, warps per block, rows per lane, fused
or separate spectrum and comb kernels, overlapped windows, the event count
from which pixels take the hybrid grid route) by the wall time
of the whole call (CUDA events on its stream), keeps the fastest, sets it on
the context, and caches the choice in a JSON file keyed by device, sensor,
grid, parameters and workload shape, so later runs reuse it without timing. Only the launch configuration changes; every
candidate computes the same per-pixel results up to FP32 summation order.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics

import torch

from . import ddhf

DEFAULT_CANDIDATES = [
    dict(heavy_min=hm, warps_per_block=wpb, blocks_per_sm=0, rows_per_lane=r, fuse=1, overlap=0)
    for hm in (512, 1024, 4096)
    for wpb in (4, 8)
    for r in (0, 4)
] + [
    dict(heavy_min=hm, warps_per_block=wpb, blocks_per_sm=0, rows_per_lane=r, fuse=0, overlap=ov,
         hybrid_min=hy)
    for hm in (128, 256, 1024, 4096)
    for wpb in (4, 8)
    for r in (0, 4)
    for ov in (0, 1)
    for hy in (0, 64, 128, 256)
]


def workload_key(ctx: "ddhf.Context", windows) -> str:
    dev = torch.cuda.get_device_name()
    g = ctx.grid
    p = ctx.params
    ev = sorted(int(w[4]) for w in windows)
    sig = dict(device=dev, W=ctx.W, H=ctx.H, grid=[g.a0, g.da, g.denom, g.n_bins],
               params=[p.tau_sf, p.tau_comb, p.M, p.d, p.h_min, p.n_min, p.A_min, p.alpha],
               windows=len(windows), events_bucket=[e >> 20 for e in ev])
    return hashlib.sha1(json.dumps(sig, sort_keys=True).encode()).hexdigest()[:16]


def _time_call(ctx, windows, boxes, cap, nbox, reps):
    """Median wall time (CUDA events on the stream) of the whole batched call;
    the first, capturing call is not counted."""
    ms = []
    for _ in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        ddhf.ddhf_detect_batch(ctx.h, windows, boxes, cap, nbox, None, use_graph=True)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms[1:])


def autotune(ctx: "ddhf.Context", windows, boxes, cap, nbox, candidates=None, reps=2,
             cache_path=None, force=False):
    """Pick the fastest tuning for these windows; returns (tuning, timings)."""
    cands = candidates or DEFAULT_CANDIDATES
    key = workload_key(ctx, windows)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if not force and key in cache:
        best = cache[key]["tuning"]
        ctx.set_tuning(**best)
        return best, cache[key].get("timings", {})
    timings = {}
    best, best_ms = None, None
    for cand in cands:
        try:
            ctx.set_tuning(**cand)
            ms = _time_call(ctx, windows, boxes, cap, nbox, reps)
        except ddhf.DDHFError:
            continue  # a candidate that does not fit (shared memory) is skipped
        timings[json.dumps(cand, sort_keys=True)] = ms
        if best_ms is None or ms < best_ms:
            best, best_ms = cand, ms
    if best is None:
        raise RuntimeError("no tuning candidate could be launched")
    ctx.set_tuning(**best)
    if cache_path:
        cache[key] = dict(tuning=best, call_ms=best_ms, timings=timings)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return best, timings
