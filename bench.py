#!/usr/bin/env python
"""Benchmark of the DDHF hot path on the 1280x720 batched workload.

One step = one ddhf_detect_batch call over 8 consecutive 30 ms windows x 4
independent event streams (32 windows, ~20M events each, 750 bins 0-1498 Hz),
replayed as one CUDA graph: per window, binning, the blocked NDFT spectrum
kernel, the spectral-flatness + comb kernel, labelling and boxes (or, with
the fused tuning, one persistent NDFT + comb kernel over all windows). The
autotuner picks the tuning first. Inputs are resident in HBM when the timed
region starts (8.3 GB per step, far above L2, so no flush is needed).

Metric: NDFT event-bin terms per second (terms = sum over active pixels of
event count x bins, the work of Eq. 6), whole job over all ranks; also
ms per window. Extra keys: roofline of the NDFT kernel (FP32 FMA-pipe bound),
e2e through the C ABI from pinned host buffers, the plain one-warp-per-pixel
pipeline on the same windows, and the FP64 oracle timed on a sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--sensor WxH runs the same recipe on a smaller sensor (profiling captures
only; the headline workload is 1280x720).

The `slide` object times the sliding window (Sec. 3.3: the terms of the
events that enter and leave a window that advances 3.75 ms per push) on the
first C3 stream; --only-slide runs just that leg (for launch-list captures),
--slide-warm sets its untimed passes.

Under torchrun every rank runs its own 32 windows (seeded by rank; weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_08386_gb300 import synth  # noqa: E402

N_STREAMS, N_WINDOWS = 4, 8
METRIC = "NDFT event-bin terms/s (1280x720, 8 windows x 4 streams per CUDA-graph launch)"
UNIT = "terms/s"
WORKLOAD = ("C3: {W}x{H}, 8 consecutive 30 ms windows x 4 streams per step, Pareto(1.5) "
            "per-pixel counts capped at 20k, 3 drones; grid 0-1498 Hz step 2 Hz (750 bins); "
            "Table 2 parameters")
OPS_PER_TERM = 3  # FP32 FMA-pipe lane-ops per term of the blocked three-multiplication form
# DRAM bytes (read + write) per active pixel of one launch, from one ncu capture
# of the kernel on a 640x360 window of the same recipe (profiles/), scaled to a
# launch by its active pixels (the traffic is per-pixel rows). A figure is
# listed only while the kernel is the one that was captured.
TRAFFIC_PER_PIXEL = {"k_comb<2>": 3044.0, "k_blocked<6,1,0>": 2894.0}
TRAFFIC_NOTE = ("null: the ncu DRAM capture of this kernel predates its current code "
                "(profiles/ keeps the earlier figure)")


def _gen_window(args):
    seed, s, w, W, H = args
    sc = synth.config3_window(s, w, seed=seed, W=W, H=H)
    return sc.x, sc.y, sc.t, sc.p, sc.t0, sc.window_us, sc.n


def _gen_c4(b):
    # window b of the soft-comb batch (640x480, 40 ms, 750 bins), as config4_batch makes it
    sc = synth.config2(1004 * 1000 + b, W=640, H=480, window_us=40_000,
                       grid=synth.hz_grid(0, 2, 750))
    return sc.x, sc.y, sc.t, sc.p, sc.t0, sc.window_us, sc.n


# thresholds inside Table 2's ranges that separate synthetic drones from the C3
# noise (Table 2's own tau_sf and tau_comb flag most noise pixels of these
# dense windows, so detection there yields one sensor-wide box)
LABELLED_PARAMS = dict(tau_sf=0.5, tau_comb=2.0, M=4, d=3, h_min=4, n_min=6, A_min=25,
                       alpha=2.0)
LABELLED_SEEDS = (400, 302, 401)


def _gen_labelled(seed):
    # a full-size labelled window: the C3 noise recipe with 1-3 drones
    s = synth.labelled_scene(seed, W=1280, H=720, min_sep=100)
    return (s.x, s.y, s.t, s.p, s.t0, s.window_us, s.n,
            [d["box"] for d in s.drones if d["box"] is not None])


def _iou(a, b):
    ix = min(a[2], b[2]) - max(a[0], b[0]) + 1
    iy = min(a[3], b[3]) - max(a[1], b[1]) + 1
    if ix <= 0 or iy <= 0:
        return 0.0
    inter = ix * iy
    area = lambda r: (r[2] - r[0] + 1) * (r[3] - r[1] + 1)
    return inter / (area(a) + area(b) - inter)


def labelled_leg(scenes, W, H, grid, tuning, torch, ddhf, replays=100):
    """Detection on full-size labelled windows (synth.labelled_scene) with
    thresholds that separate the drones: the graph-replayed one-window call
    timed replay by replay, and what it found (boxes, rotor pixels, ground-truth
    drones matched at IoU >= 0.5, the paper's matching rule)."""
    rows = []
    for (x, y, t, p, t0, win, n, gt) in scenes:
        c = ddhf.Context(W, H, grid, ddhf.default_params(**LABELLED_PARAMS), max_events=max(n, 1),
                         max_windows=1)
        c.set_tuning(**{k: v for k, v in tuning.items() if k != "how"})
        d = [torch.from_numpy(a).cuda() for a in (x, y, t, p)]
        wl = [(d[0], d[1], d[2], d[3], n, t0, win)]
        bx = torch.empty((256, 5), dtype=torch.int32, device="cuda")
        nb = torch.zeros(1, dtype=torch.int32, device="cuda")
        for _ in range(5):
            ddhf.ddhf_detect_batch(c.h, wl, bx, 256, nb, None, use_graph=True)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(replays)]
        for a, b in evs:
            a.record()
            ddhf.ddhf_detect_batch(c.h, wl, bx, 256, nb, None, use_graph=True)
            b.record()
        torch.cuda.synchronize()
        lt = np.array([a.elapsed_time(b) for a, b in evs])
        k = int(nb.item())
        boxes = bx[:min(k, 256)].cpu().numpy()
        st = c.stats()
        c.close()
        matched = sum(1 for g in gt if any(_iou(g, b[:4]) >= 0.5 for b in boxes))
        true_boxes = sum(1 for b in boxes if any(_iou(g, b[:4]) >= 0.5 for g in gt))
        q25, q50, q75, q95 = np.percentile(lt, [25, 50, 75, 95])
        rows.append(dict(events=int(n), active_pixels=int(st["n_active"]),
                         rotor_pixels=int(st["n_rotor"]), boxes=k, drones=len(gt),
                         drones_matched=matched, boxes_matching_a_drone=true_boxes,
                         median_ms=float(q50), iqr_ms=float(q75 - q25), p95_ms=float(q95)))
    return dict(window=f"{W}x{H}, 30 ms labelled windows (C3 noise recipe, 1-3 drones), seeds "
                       f"{list(LABELLED_SEEDS)}; {replays} graph replays each",
                params=LABELLED_PARAMS, points=rows)


def slide_leg(wins, W, H, grid, torch, ddhf, hop_us=3750, rebuild_every=64, cap_box=256,
              warm_passes=2):
    """The sliding window on one C3 stream (consecutive windows of stream 0):
    a 30 ms window advanced by hop_us per push. The pushes that fill the first
    window are untimed; every later push (event delta of hop_us in and out)
    and the detection that follows it are timed one by one with CUDA events.
    A second pass with rebuild_every = 1 times pushes that recompute the whole
    window's state instead."""
    T, t0 = int(wins[0][5]), int(wins[0][4])
    x = np.concatenate([w[0] for w in wins])
    y = np.concatenate([w[1] for w in wins])
    t = np.concatenate([w[2] for w in wins])
    p = np.concatenate([w[3] for w in wins])
    order = np.argsort(t, kind="stable")
    x, y, t, p = x[order], y[order], t[order], p[order]
    n_hops = (len(wins) * T) // hop_us
    fill = T // hop_us
    bounds = np.searchsorted(t, t0 + hop_us * np.arange(n_hops + 1))
    per = np.diff(bounds)
    cap = int(max(per[i:i + fill + 1].sum() for i in range(n_hops)) * 1.05) + 1
    d = [torch.from_numpy(a).cuda() for a in (x, y, t, p)]
    sc = ddhf.Context(W, H, grid, max_events=cap)
    bx = torch.empty((cap_box, 5), dtype=torch.int32, device="cuda")
    nb = torch.zeros(1, dtype=torch.int32, device="cuda")

    def run(every):
        sc.slide_begin(T, t0, cap, every)
        ev, st0 = [], None
        for i in range(n_hops):
            lo, hi = int(bounds[i]), int(bounds[i + 1])
            if i == fill:
                st0 = sc.slide_stats()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            ddhf.ddhf_slide_push(sc.h, d[0][lo:hi], d[1][lo:hi], d[2][lo:hi], d[3][lo:hi],
                                 hi - lo, t0 + hop_us * (i + 1))
            e[1].record()
            ddhf.ddhf_slide_detect(sc.h, bx, cap_box, nb)
            e[2].record()
            if i >= fill:
                ev.append(e)
        st1 = sc.slide_stats()
        torch.cuda.synchronize()
        push = np.array([a.elapsed_time(b) for a, b, _ in ev])
        det = np.array([b.elapsed_time(c) for _, b, c in ev])
        delta = (st1["n_added"] - st0["n_added"]) + (st1["n_expired"] - st0["n_expired"])
        return push, det, delta, st1

    for _ in range(warm_passes):
        run(rebuild_every)
    push, det, delta, st = run(rebuild_every)
    rpush, rdet, _, _ = run(1)
    sc.stats()
    sc.close()
    nbins = grid[3]
    n = len(push)
    return dict(
        workload=f"C3 stream 0 ({W}x{H}), consecutive 30 ms windows; the window advances "
                 f"{hop_us} us per push; {n} timed pushes after the {fill} that fill it",
        window_us=T, hop_us=hop_us, rebuild_every=rebuild_every, timed_pushes=n,
        events_per_hop=float(np.mean(per[fill:])), delta_events_per_hop=delta / n,
        push_ms_median=float(np.median(push)), detect_ms_median=float(np.median(det)),
        hop_ms_median=float(np.median(push + det)),
        delta_terms_per_s=delta * nbins / (push.sum() * 1e-3),
        rebuild_push_ms_median=float(np.median(rpush)),
        amortised_hop_ms=float(np.median(push + det)
                               + (np.median(rpush) - np.median(push)) / rebuild_every),
        state_bytes=W * H * ((nbins + 31) // 32 * 32) * 8, window_events_last=st["n_window"],
        pixels_last_push=st["last_pixels"],
        # algorithmic bytes of a push: each touched pixel's state row read and
        # written (n_bins complex FP32), the delta's packed words read
        push_state_gbs=(st["last_pixels"] * nbins * 16 + delta / n * 8) / (np.median(push) * 1e-3)
        / 1e9,
        unit="ms per hop (CUDA events); delta terms = (events in + events out) x bins")


def latency_sweep(means, W, H, grid, torch, ddhf, replays=100, seed=1003):
    """One 1280x720 window of the C3 recipe at lower event densities (stream 0,
    window 0, the Pareto counts scaled to `mean` events per pixel): the
    graph-replayed detection timed replay by replay, each density with the
    tuning the autotuner picks on that window (a sparse window gains from other
    thresholds than the full-density batch: the hybrid route's fixed cost is
    not repaid by a few heavy pixels). Gives the largest event count whose
    median latency is under 1 ms."""
    from paper_2603_08386_gb300 import tune
    rows = []
    for m in means:
        sc = synth.config3_window(0, 0, seed=seed, W=W, H=H, mean_per_px=m)
        c = ddhf.Context(W, H, grid, max_events=max(sc.n, 1), max_windows=1)
        d = ddhf.events_to_device(sc)
        wl = [(d[0], d[1], d[2], d[3], sc.n, sc.t0, sc.window_us)]
        bx = torch.empty((256, 5), dtype=torch.int32, device="cuda")
        nb = torch.zeros(1, dtype=torch.int32, device="cuda")
        tun, _ = tune.autotune(c, wl, bx, 256, nb)
        for _ in range(5):
            ddhf.ddhf_detect_batch(c.h, wl, bx, 256, nb, None, use_graph=True)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(replays)]
        for a, b in evs:
            a.record()
            ddhf.ddhf_detect_batch(c.h, wl, bx, 256, nb, None, use_graph=True)
            b.record()
        torch.cuda.synchronize()
        lt = np.array([a.elapsed_time(b) for a, b in evs])
        st = c.stats()
        c.close()
        q25, q50, q75, q95 = np.percentile(lt, [25, 50, 75, 95])
        rows.append(dict(mean_per_px=m, events=int(sc.n), active_pixels=int(st["n_active"]),
                         terms=int(st["terms"]), median_ms=float(q50), iqr_ms=float(q75 - q25),
                         p95_ms=float(q95), tuning=tun))
    under = [r["events"] for r in rows if r["median_ms"] < 1.0]
    return dict(window=f"{W}x{H}, 30 ms, C3 recipe (stream 0, window 0) at lower densities; "
                       f"{replays} graph replays each, autotuned per density",
                points=rows, largest_events_under_1ms=max(under) if under else None)


def rank_seed(rank: int) -> int:
    """Seed of a rank's batch: ranks are independent replicas (weak scaling)."""
    return 1003 + 1000 * rank


def max_over_ranks(value: float, dist, device) -> float:
    """Slowest rank's value (the job time), via an all-reduce MAX."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(terms_per_rank_step: int, world: int, steps: int, ms_max: float) -> float:
    """Whole-job terms/s: every rank processed terms_per_rank_step per step."""
    return terms_per_rank_step * world * steps / (ms_max * 1e-3)


def generate(rank: int, procs: int, n_windows: int = N_STREAMS * N_WINDOWS, W: int = 1280,
             H: int = 720):
    seed = rank_seed(rank)
    jobs = [(seed, s, w, W, H) for s in range(N_STREAMS) for w in range(N_WINDOWS)][:n_windows]
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=max(1, min(procs, len(jobs)))) as pool:
        return pool.map(_gen_window, jobs, chunksize=1)


def _counts(win, W, H):
    x, y, t, p, t0, wus, n = win
    ok = (x >= 0) & (x < W) & (y >= 0) & (y < H) & (t >= t0) & (t < t0 + wus) & (p != 0)
    return np.bincount(y[ok].astype(np.int64) * W + x[ok], minlength=W * H)


def terms_of(win, W, H, n_bins, n_min=6):
    cnt = _counts(win, W, H)
    return int(cnt[cnt >= n_min].sum()) * n_bins


def active_of(win, W, H, n_min=6):
    return int((_counts(win, W, H) >= n_min).sum())


def measured_peaks():
    """Measured peaks of this GPU pool, else the recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured")
    except (OSError, ValueError, KeyError):
        return dict(hbm_gbs=6800.0, source="fallback")


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.path = os.path.join("/tmp", f"ddhf_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                       f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [v.strip() for v in line.split(",")]
            if len(parts) >= 7:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"])

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0])]
        smax = [num(r[1]) for r in rows if num(r[1])]
        power = [num(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i] == "Active"})
        load = [v for v in sm if v >= 0.5 * max(sm)] if sm else []
        return dict(sm_mhz=statistics.median(load) if load else None,
                    sm_max_mhz=max(smax) if smax else None, reasons=reasons,
                    samples=len(rows), power_w_max=max(power) if power else None)


def oracle_bin(win, W, H):
    import oracle
    x, y, t, p, t0, wus, n = win
    return oracle.bin_events(W, H, x, y, t, p, t0, wus)


def oracle_sample(b, W, H, grid, n_pixels, seed=5):
    """FP64 oracle (as it stands) on a seeded sample of one binned window's
    active pixels: per-pixel NDFT + SF + comb (Eq. 6-11).
    Returns (terms, seconds, pixels)."""
    import oracle
    act = np.flatnonzero(b["counts"] >= 6)
    rng = np.random.default_rng(seed)
    pix = np.sort(rng.choice(act, size=min(n_pixels, act.size), replace=False))
    terms = int(b["counts"][pix].sum()) * grid[3]
    t_0 = time.perf_counter()
    oracle.classify(W, H, b, grid, pixels=pix)
    return terms, time.perf_counter() - t_0, int(pix.size)


def _oracle_chunk(args):
    """One worker's share of the CPU baseline: the oracle, as it stands, on a
    list of active pixels (Eq. 6-11 per pixel), given as a one-row sensor that
    holds just those pixels' events (so that little is sent to the worker)."""
    import oracle
    npx, b, grid = args
    t_0 = time.perf_counter()
    oracle.classify(npx, 1, b, grid)
    return time.perf_counter() - t_0


def _oracle_chunk_f32(args):
    """One worker's share of the FP32 CPU baseline: the oracle's FP32 NDFT
    (Eq. 6 in single precision) of each pixel of the subset."""
    import oracle
    npx, b, grid = args
    t_0 = time.perf_counter()
    offs = b["offsets"]
    for k in range(npx):
        oracle.ndft_f32(b["tau"][offs[k]:offs[k + 1]], b["pol"][offs[k]:offs[k + 1]], *grid)
    return time.perf_counter() - t_0


def _pixel_subset(b, pix):
    """The events of pixels `pix` of a binned window as a one-row sensor."""
    cnt = b["counts"][pix]
    offs = np.zeros(pix.size + 1, np.int64)
    offs[1:] = np.cumsum(cnt)
    sel = np.concatenate([np.arange(b["offsets"][k], b["offsets"][k + 1]) for k in pix])
    return dict(offsets=offs, tau=b["tau"][sel], pol=b["pol"][sel], counts=cnt)


def oracle_all_cores(b, W, H, grid, n_pixels, seed=5, procs=None, fp32_ndft=False):
    """The oracle on a seeded sample of active pixels split over every host
    core (one spawned worker per core, each a single-threaded oracle call):
    Eq. 6-11 in FP64, or (fp32_ndft) the FP32 NDFT alone.
    Returns (terms, wall seconds, pixels, workers)."""
    work = _oracle_chunk_f32 if fp32_ndft else _oracle_chunk
    procs = procs or os.cpu_count() or 1
    act = np.flatnonzero(b["counts"] >= 6)
    rng = np.random.default_rng(seed)
    pix = np.sort(rng.choice(act, size=min(n_pixels, act.size), replace=False))
    terms = int(b["counts"][pix].sum()) * grid[3]
    chunks = [c for c in np.array_split(pix, procs) if c.size]
    jobs = [(c.size, _pixel_subset(b, c), grid) for c in chunks]
    with mp.get_context("spawn").Pool(processes=len(chunks)) as pool:
        pool.map(work, [(1, _pixel_subset(b, chunks[0][:1]), grid)] * len(chunks))
        t_0 = time.perf_counter()
        pool.map(work, jobs, chunksize=1)
        wall = time.perf_counter() - t_0
    return terms, wall, int(pix.size), len(chunks)


def run_reference(args):
    """The oracle timed on the host cores on bounded samples of the workload:
    each step scores a seeded sample of active pixels of one C3 window with
    one spawned single-threaded oracle worker per host core."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc = synth.config3_window(0, 0)
    b = oracle_bin((sc.x, sc.y, sc.t, sc.p, sc.t0, sc.window_us, sc.n), sc.W, sc.H)
    procs = os.cpu_count() or 1
    per_step = 40 * procs
    act = np.flatnonzero(b["counts"] >= 6)
    tot_terms, tot_s = 0, 0.0
    with mp.get_context("spawn").Pool(processes=procs) as pool:
        for i in range(args.warmup + args.steps):
            rng = np.random.default_rng(1000 + i)
            pix = np.sort(rng.choice(act, size=min(per_step, act.size), replace=False))
            jobs = [(c.size, _pixel_subset(b, c), sc.grid)
                    for c in np.array_split(pix, procs) if c.size]
            t_0 = time.perf_counter()
            pool.map(_oracle_chunk, jobs, chunksize=1)
            dt = time.perf_counter() - t_0
            if i >= args.warmup:
                tot_terms += int(b["counts"][pix].sum()) * sc.grid[3]
                tot_s += dt
    v = tot_terms / tot_s
    sample = (f"per step {per_step} seeded random active pixels of window 0 of stream 0 "
              f"(1280x720, 750 bins), split over {procs} spawned single-threaded oracle "
              f"workers: FP64 NDFT + SF + comb")
    line = dict(impl="reference", metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * tot_s / args.steps,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic",
                config=dict(workload=WORKLOAD.format(W=1280, H=720),
                            sample="oracle on seeded pixel samples of window 0 of stream 0"),
                cpu_baseline=dict(value=v, unit=UNIT, cores=procs, kind="oracle", sample=sample),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-pipeline comparison")
    ap.add_argument("--no-oracle", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer e2e loop")
    ap.add_argument("--windows", type=int, default=N_STREAMS * N_WINDOWS,
                    help="windows per step (default 32; fewer only for profiling cases)")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default tuning)")
    ap.add_argument("--tuning", default=None,
                    help="JSON dict of ddhf_tuning fields to use instead of the autotuner")
    ap.add_argument("--procs", type=int, default=int(os.environ.get("DDHF_GEN_PROCS", "16")))
    ap.add_argument("--no-latency", action="store_true", help="skip the one-window latency")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the one-window latency at lower event densities")
    ap.add_argument("--no-softcomb", action="store_true", help="skip the soft-comb timing")
    ap.add_argument("--no-labelled", action="store_true",
                    help="skip the detection on labelled windows")
    ap.add_argument("--no-slide", action="store_true", help="skip the sliding-window timing")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the one-window blocked / hybrid spectrum timing")
    ap.add_argument("--only-slide", action="store_true",
                    help="run only the sliding-window leg and print its object (profiling)")
    ap.add_argument("--slide-warm", type=int, default=2, help="untimed sliding-window passes")
    ap.add_argument("--softcomb-windows", type=int, default=16)
    ap.add_argument("--latency-replays", type=int, default=100)
    ap.add_argument("--sensor", default="1280x720",
                    help="WxH of the synthetic sensor (smaller sizes for profiling captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    W, H = (int(v) for v in args.sensor.lower().split("x"))
    # inputs are generated before any CUDA call (spawned workers)
    wins = generate(rank, max(1, args.procs // max(1, world)), args.windows, W, H)
    c4 = []
    if not args.no_softcomb and args.softcomb_windows > 0:
        with mp.get_context("spawn").Pool(processes=max(1, min(args.procs,
                                                                  args.softcomb_windows))) as pool:
            c4 = pool.map(_gen_c4, range(args.softcomb_windows))
    lab = []
    if not args.no_labelled and rank == 0 and (W, H) == (1280, 720):
        with mp.get_context("spawn").Pool(processes=len(LABELLED_SEEDS)) as pool:
            lab = pool.map(_gen_labelled, LABELLED_SEEDS)

    import torch
    from paper_2603_08386_gb300 import build, ddhf
    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    grid = synth.hz_grid(0, 2, 750)
    nb = grid[3]
    if args.only_slide:
        if rank == 0:
            print(json.dumps(dict(slide=slide_leg(wins[:2], W, H, grid, torch, ddhf,
                                                  warm_passes=args.slide_warm))), flush=True)
        return
    terms_step = sum(terms_of(w, W, H, nb) for w in wins)
    events_step = sum(w[6] for w in wins)
    max_ev = max(w[6] for w in wins)
    nwin = len(wins)
    cap = 256
    ctx = ddhf.Context(W, H, grid, max_events=max_ev, max_windows=nwin)
    dev = [tuple(torch.from_numpy(a).cuda() for a in w[:4]) for w in wins]
    wl = [(d[0], d[1], d[2], d[3], w[6], w[4], w[5]) for d, w in zip(dev, wins)]
    boxes = torch.empty((nwin * cap, 5), dtype=torch.int32, device="cuda")
    nbox = torch.zeros(nwin, dtype=torch.int32, device="cuda")
    # pipe throughput of this device (the NDFT roofline's denominator), before
    # the workload's first launch
    peaks = ddhf.ddhf_measure_pipes()
    tuning, tune_note = ddhf.ddhf_get_tuning(ctx.h), "default"
    if args.tuning:
        ctx.set_tuning(**json.loads(args.tuning))
        tuning, tune_note = ddhf.ddhf_get_tuning(ctx.h), "given on the command line"
    elif not args.no_tune:
        # the autotuner times the whole batched call on the first 4 windows of this batch
        from paper_2603_08386_gb300 import tune
        k = min(4, nwin)
        tctx = ddhf.Context(W, H, grid, max_events=max_ev, max_windows=k)
        tb = torch.empty((k * cap, 5), dtype=torch.int32, device="cuda")
        tn = torch.zeros(k, dtype=torch.int32, device="cuda")
        tuning, _ = tune.autotune(tctx, wl[:k], tb, cap, tn)
        tctx.close()
        ctx.set_tuning(**tuning)
        tune_note = f"autotuned on {k} windows"

    def step():
        ddhf.ddhf_detect_batch(ctx.h, wl, boxes, cap, nbox, None, use_graph=True)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    st = ctx.stats()
    graph_kernels = st["graph_kernels"]
    # ------------------------------------------------------------ timed region
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    ms_step = ms / args.steps
    value = job_throughput(terms_step, world, args.steps, ms)
    st = ctx.stats()
    # ------------------------------------------------------------ per-stage breakdown
    # after the timed region: the same step with CUDA events around each stage
    # (a separately captured graph; each step is read back before the next)
    ddhf.ddhf_enable_stage_timing(ctx.h, True)
    step()
    torch.cuda.synchronize()
    fused_ms, bin_ms, box_ms, spec_ms, comb_ms = [], [], [], [], []
    for _ in range(3):
        step()
        b_ms, f_ms, x_ms, sp_ms, cb_ms = ddhf.ddhf_stage_times(ctx.h)
        bin_ms.append(b_ms)
        fused_ms.append(f_ms)
        box_ms.append(x_ms)
        spec_ms.append(sp_ms)
        comb_ms.append(cb_ms)
    ddhf.ddhf_enable_stage_timing(ctx.h, False)
    # ------------------------------------------------------------ e2e from pinned host memory
    e2e = None
    if not args.no_e2e:
        host = [tuple(torch.from_numpy(a).pin_memory() for a in w[:4]) for w in wins]
        h2d = sum(sum(a.numel() * a.element_size() for a in hw) for hw in host)
        hbox = torch.empty((nwin * cap, 5), dtype=torch.int32).pin_memory()
        hn = torch.empty(nwin, dtype=torch.int32).pin_memory()
        d2h = hbox.numel() * 4 + hn.numel() * 4

        hwins = [(hw[0], hw[1], hw[2], hw[3], w[6], w[4], w[5]) for hw, w in zip(host, wins)]

        def e2e_step():
            # the library call on host buffers: each window's events are copied
            # while the previous window is processed; boxes come back to host
            ddhf.ddhf_detect_batch_host(ctx.h, hwins, hbox, cap, hn)

        e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e2e_steps = max(1, min(args.steps, 5))
        e0.record()
        for _ in range(e2e_steps):
            e2e_step()
        e1.record()
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        # the host-to-device copies alone (same pinned buffers, one stream):
        # the bandwidth that bounds the end-to-end rate when it is below the
        # step's own rate
        dst = [tuple(torch.empty_like(a, device="cuda") for a in hw) for hw in host]
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        for hw, dw in zip(host, dst):
            for a, b_ in zip(hw, dw):
                b_.copy_(a, non_blocking=True)
        c1.record()
        torch.cuda.synchronize()
        h2d_ms = c0.elapsed_time(c1)
        del dst
        e2e = dict(value=job_throughput(terms_step, world, e2e_steps, e2e_ms), unit=UNIT,
                   h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h, steps=e2e_steps,
                   ms_per_step=e2e_ms / e2e_steps, h2d_alone_ms_per_step=h2d_ms,
                   h2d_alone_gbs=h2d / (h2d_ms * 1e-3) / 1e9,
                   call="ddhf_detect_batch_host (pinned host events in, host boxes out)")
    # ------------------------------------------------------------ one-window latency
    # a single 1280x720 window (stream 0, window 0) through the graph-replayed
    # detection call, each replay timed on its own, after the bench's tuning
    lat = None
    if not args.no_latency:
        lc = ddhf.Context(W, H, grid, max_events=max_ev, max_windows=1)
        lc.set_tuning(**{k: v for k, v in tuning.items() if k != "how"})
        lb = torch.empty((cap, 5), dtype=torch.int32, device="cuda")
        ln = torch.zeros(1, dtype=torch.int32, device="cuda")
        for _ in range(5):
            ddhf.ddhf_detect_batch(lc.h, wl[:1], lb, cap, ln, None, use_graph=True)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.latency_replays)]
        for a, b in evs:
            a.record()
            ddhf.ddhf_detect_batch(lc.h, wl[:1], lb, cap, ln, None, use_graph=True)
            b.record()
        torch.cuda.synchronize()
        lt = np.array([a.elapsed_time(b) for a, b in evs])
        q25, q50, q75, q95 = np.percentile(lt, [25, 50, 75, 95])
        lat = dict(window="stream 0, window 0 (one 30 ms window of the batch)",
                   events=int(wins[0][6]), replays=len(lt), median_ms=float(q50),
                   iqr_ms=float(q75 - q25), p95_ms=float(q95), min_ms=float(lt.min()))
        lc.close()
    # ------------------------------------------------------------ latency at lower densities
    sweep = None
    if not args.no_sweep and rank == 0:
        sweep = latency_sweep((1.0, 2.0, 3.0, 5.0, 10.0), W, H, grid, torch, ddhf,
                              replays=args.latency_replays)
    labelled = None
    if lab:
        labelled = labelled_leg(lab, W, H, grid, tuning, torch, ddhf, replays=args.latency_replays)
        del lab
    # ------------------------------------------------------------ spectrum forms, one window
    # window 0 alone through ddhf_power_spectrum: the blocked kernel on every
    # active pixel (the FMA-pipe roofline of that kernel, without the hybrid
    # split) and the hybrid form, whose heavy pixels take the uniform-grid
    # route (spread + dense product with the shared table)
    forms = None
    if not args.no_forms:
        fc = ddhf.Context(W, H, grid, max_events=max_ev, max_windows=1)
        d0, w0 = dev[0], wins[0]
        ddhf.ddhf_bin_events(fc.h, d0[0], d0[1], d0[2], d0[3], w0[6], w0[4], w0[5])
        na0 = fc.n_active()
        P0 = torch.empty((max(na0, 1), nb), dtype=torch.float32, device="cuda")
        hm = int(tuning.get("hybrid_min", 0)) or 64
        base = {k: v for k, v in tuning.items() if k != "how"}
        forms = dict(window="stream 0, window 0", active_pixels=na0,
                     terms=terms_of(w0, W, H, nb))
        # the blocked kernel alone takes every pixel, so its own heavy threshold
        # (block-per-pixel from heavy_min events) is chosen here among a few
        # values; the step's tuning picks heavy_min for the pixels that the
        # hybrid route leaves to it
        runs = [("blocked", ddhf.FORM["blocked"], dict(base, hybrid_min=0, heavy_min=h))
                for h in sorted({128, 256, 512, 1024, int(base.get("heavy_min", 1024))})]
        runs.append(("hybrid", ddhf.FORM["hybrid"], dict(base, hybrid_min=hm)))
        for name, form, tun in runs:
            fc.set_tuning(**tun)
            for _ in range(3):
                ddhf.ddhf_power_spectrum(fc.h, form, P0, na0)
            torch.cuda.synchronize()
            fe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(10)]
            for a_, b_ in fe:
                a_.record()
                ddhf.ddhf_power_spectrum(fc.h, form, P0, na0)
                b_.record()
            torch.cuda.synchronize()
            ms_ = float(np.median([a_.elapsed_time(b_) for a_, b_ in fe]))
            if name == "hybrid":
                forms["hybrid_ms"] = ms_
            else:
                forms.setdefault("blocked_by_heavy_min", {})[str(tun["heavy_min"])] = ms_
                if ms_ < forms.get("blocked_ms", float("inf")):
                    forms["blocked_ms"], forms["blocked_heavy_min"] = ms_, tun["heavy_min"]
        fc.stats()
        fc.close()
        cnt0 = _counts(w0, W, H)
        s_us = grid[2] // (2 * grid[1] * nb)
        G = (int(w0[5]) - 1) // s_us + 8 if s_us >= 1 else 0
        thr = max(hm, 16, -(-G // 2))
        hv = cnt0[cnt0 >= thr] if 16 <= G <= 1024 else cnt0[:0]
        forms.update(hybrid_min=hm, grid_spacing_us=int(s_us), grid_rows=int(G),
                     threshold=int(thr), hybrid_pixels=int(hv.size),
                     hybrid_events=int(hv.sum()),
                     blocked_tops=OPS_PER_TERM * forms["terms"] / (forms["blocked_ms"] * 1e-3)
                     / 1e12,
                     note="hybrid pixels: G grid values each instead of their events")
    # ------------------------------------------------------------ sliding window
    slide = None
    if not args.no_slide and nwin >= 2:
        slide = slide_leg(wins[:2], W, H, grid, torch, ddhf, warm_passes=args.slide_warm)
        if lat:
            slide["full_window_ms_median"] = lat["median_ms"]
    # ------------------------------------------------------------ soft comb and its adjoint
    # C4: a batch of 640x480 windows (16 by default) laid out as one window of
    # a 640 x (16 * 480) sensor (ddhf.stack_windows), binned once; one
    # ddhf_softcomb call scores every active pixel of the batch (S), one more
    # gives dS/d(f0, w, sigma), for 6 harmonics x (2Q+1) = 42 evaluation
    # frequencies per pixel
    softc = None
    if c4:
        Q, delta, n_h = 3, 2.0, 6
        nwc = len(c4)
        w4 = c4[0][5]
        xs, ys, ts, ps = ddhf.stack_windows([(a[0], a[1], a[2], a[3], a[4]) for a in c4], 480)
        n4 = int(xs.size)
        cc = ddhf.Context(640, 480 * nwc, grid, max_events=n4)
        d4 = [torch.from_numpy(a).cuda() for a in (xs, ys, ts, ps)]
        cc.bin_events(*d4, 0, w4)
        csr = cc.csr()
        pix = csr["active"]
        na = pix.numel()
        offs = csr["offsets"].long()
        cnt = int((offs[pix.long() + 1] - offs[pix.long()]).sum().item())
        gen = torch.Generator(device="cuda").manual_seed(1004)
        f0 = 50.0 + 150.0 * torch.rand(na, device="cuda", generator=gen)
        wv = torch.ones(n_h, device="cuda")
        sg = torch.full((n_h,), 2.0, device="cuda")
        Bv = torch.ones(na, device="cuda")
        Sv = torch.empty(na, device="cuda")
        gS = torch.ones(na, device="cuda")
        gf, gw, gsg = torch.empty(na, device="cuda"), torch.empty(n_h, device="cuda"), \
            torch.empty(n_h, device="cuda")
        fwd = lambda: ddhf.ddhf_softcomb(cc.h, pix, f0, n_h, Q, delta, w4 / 2, wv, sg, Bv, S=Sv)
        bwd = lambda: ddhf.ddhf_softcomb(cc.h, pix, f0, n_h, Q, delta, w4 / 2, wv, sg, Bv,
                                         grad_S=gS, grad_f0=gf, grad_w=gw, grad_sigma=gsg)
        timed = {}
        for name, fn in (("fwd", fwd), ("bwd", bwd)):
            fn()
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record()
            for _ in range(5):
                fn()
            a1.record()
            torch.cuda.synchronize()
            timed[name] = a0.elapsed_time(a1) / 5
        cc.stats()
        cc.close()
        del d4
        terms_sc = cnt * n_h * (2 * Q + 1)
        softc = dict(workload=f"C4: {nwc} windows of 640x480, 40 ms (C2 density), 750-bin grid, "
                              "stacked into one 640x" + str(480 * nwc) + " window; every active "
                              "pixel; 6 harmonics, Q=3, delta 2 Hz; one call per direction",
                     windows=nwc, events=n4, pixels=na, terms=terms_sc,
                     fwd_ms_per_call=timed["fwd"], bwd_ms_per_call=timed["bwd"],
                     fwd_ms_per_window=timed["fwd"] / nwc,
                     bwd_ms_per_window=timed["bwd"] / nwc,
                     fwd_terms_per_s=terms_sc / (timed["fwd"] * 1e-3),
                     bwd_terms_per_s=terms_sc / (timed["bwd"] * 1e-3),
                     unit="event x evaluation-frequency terms/s")
    # ------------------------------------------------------------ plain per-pixel pipeline
    plain = None
    if not args.no_plain:
        pc = ddhf.Context(W, H, grid, max_events=max_ev, max_windows=1)
        k = min(4, nwin)
        P = torch.empty((W * H, nb), dtype=torch.float32, device="cuda")
        lsf = torch.empty(W * H, device="cuda")
        snr = torch.empty(W * H, device="cuda")
        f0 = torch.empty(W * H, dtype=torch.int32, device="cuda")
        mask = torch.empty(W * H, dtype=torch.uint8, device="cuda")
        lab = torch.empty(W * H, dtype=torch.int32, device="cuda")
        pb = torch.empty((cap, 5), dtype=torch.int32, device="cuda")
        pn = torch.zeros(1, dtype=torch.int32, device="cuda")

        def plain_window(i):
            d, w = dev[i], wins[i]
            ddhf.ddhf_bin_events(pc.h, d[0], d[1], d[2], d[3], w[6], w[4], w[5])
            ddhf.ddhf_power_spectrum(pc.h, ddhf.FORM["recur"], P, W * H)
            ddhf.ddhf_comb_score(pc.h, P, W * H, lsf, snr, f0, mask)
            ddhf.ddhf_label(pc.h, mask, lab)
            ddhf.ddhf_boxes(pc.h, lab, pb, cap, pn)

        plain_window(0)
        torch.cuda.synchronize()
        e0.record()
        for i in range(k):
            plain_window(i)
        e1.record()
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / k
        pterms = sum(terms_of(wins[i], W, H, nb) for i in range(k)) / k
        plain = dict(form="recur, one warp per pixel, per-window launches, spectra in HBM",
                     ms_per_window=pms, value=pterms / (pms * 1e-3), unit=UNIT,
                     windows=k)
        pc.close()
    # ------------------------------------------------------------ CPU baseline (oracle)
    cpu = None
    if rank == 0 and world == 1 and not args.no_oracle:
        b0 = oracle_bin(wins[0], W, H)
        ncores = os.cpu_count() or 1
        tr, secs, npix, nw = oracle_all_cores(b0, W, H, grid, 400 * ncores)
        tr1, secs1, npix1 = oracle_sample(b0, W, H, grid, 600, seed=6)
        cpu = dict(value=tr / secs, unit=UNIT, cores=nw, kind="oracle",
                   sample=f"{npix} seeded random active pixels of window 0 of stream 0, split "
                          f"over {nw} spawned single-threaded oracle workers (one per host "
                          f"core): FP64 NDFT + SF + comb (Eq. 6-11), {secs:.1f} s wall",
                   one_core=dict(value=tr1 / secs1, pixels=npix1, seconds=secs1),
                   host_cores=ncores)
        tr2, secs2, npix2, nw2 = oracle_all_cores(b0, W, H, grid, 3000 * ncores, seed=7,
                                                  fp32_ndft=True)
        cpu["fp32_ndft"] = dict(value=tr2 / secs2, unit=UNIT, cores=nw2,
                                sample=f"{npix2} seeded random active pixels of window 0, "
                                       f"{nw2} spawned workers: the oracle's FP32 NDFT (Eq. 6 "
                                       f"alone, single precision), {secs2:.1f} s wall")
    f_avg = statistics.mean(fused_ms)
    fused_mode = statistics.mean(spec_ms) == 0.0
    peak = peaks["ffma2_lane_per_s"] / 1e12
    hybrid_on = not fused_mode and int(tuning.get("hybrid_min", 0)) > 0
    if fused_mode:
        ndft_ms, kern = f_avg, "fused blocked NDFT + SF + comb kernel (k_blocked<TB,NW,1>)"
    else:
        ndft_ms, kern = statistics.mean(spec_ms), "blocked NDFT spectrum kernel (k_blocked<TB,1,0>)"
    achieved = OPS_PER_TERM * terms_step / (ndft_ms * 1e-3) / 1e12
    ndft_launches, ndft_launch_ms = nwin, ndft_ms / nwin
    if hybrid_on and forms:
        # the step's spectrum stage runs the blocked and the hybrid kernels; the
        # blocked kernel's own rate comes from the one-window FORM_BLOCKED run
        kern = ("blocked NDFT spectrum kernel (k_blocked<TB,1,0>) on every active pixel of "
                "one window (ddhf_power_spectrum, FORM_BLOCKED)")
        achieved = forms["blocked_tops"]
        ndft_launches, ndft_launch_ms = 1, forms["blocked_ms"]
    elif hybrid_on:
        kern += " with the hybrid grid kernels (spectrum stage time)"
    n_act = sum(active_of(w, W, H) for w in wins)
    tb = 6 if nb <= 768 and nb > 512 else None  # rows per lane the launcher picks for 750 bins
    # the captured traffic is that of the blocked kernel on every active pixel
    blocked_alone = not fused_mode and (not hybrid_on or bool(forms))
    tr_ndft = (TRAFFIC_PER_PIXEL["k_blocked<6,1,0>"] * n_act / nwin
               if ("k_blocked<6,1,0>" in TRAFFIC_PER_PIXEL and blocked_alone and tb == 6
                   and int(tuning.get("rows_per_lane", 0)) in (0, 6))
               else None)
    roof_ndft = dict(bound="alu", achieved=achieved, peak=peak, unit="Tops/s",
                     frac=achieved / peak, traffic=tr_ndft, traffic_unit="B per launch (window)",
                     traffic_note=None if tr_ndft is not None else TRAFFIC_NOTE,
                     kernel=kern, launches_per_step=ndft_launches, launch_ms=ndft_launch_ms,
                     kernel_ms_per_step=ndft_ms, share_of_step=ndft_ms / ms_step,
                     peak_source=("measured: ddhf_measure_pipes, paired FP32 FMA (f32x2) "
                                  f"chains on {peaks['sm_count']} SMs"),
                     ops="3 FP32 FMA-pipe lane-ops per term (three-multiplication complex "
                         "product)")
    roof_comb = None
    comb_reg = 512 < nb <= 768  # Table 2's M = 4, d = 3 on this grid: the register form
    if not fused_mode:
        pk = measured_peaks()
        # algorithmic bytes: read every active pixel's spectrum row, write its
        # four results (4 + 4 + 4 + 1 B), clear the window's mask
        comb_bytes = n_act * (nb * 4 + 13) + nwin * W * H
        comb_t = statistics.mean(comb_ms)
        ach = comb_bytes / (comb_t * 1e-3) / 1e9
        roof_comb = dict(bound="hbm", achieved=ach, peak=pk["hbm_gbs"], unit="GB/s",
                         frac=ach / pk["hbm_gbs"],
                         traffic=TRAFFIC_PER_PIXEL["k_comb<2>"] * n_act / nwin
                         if ("k_comb<2>" in TRAFFIC_PER_PIXEL and comb_reg) else None,
                         traffic_unit="B per launch (window)",
                         traffic_note=None if ("k_comb<2>" in TRAFFIC_PER_PIXEL and comb_reg)
                         else TRAFFIC_NOTE,
                         kernel="SF + comb kernel (k_comb<2>: register form, 24 bins per lane)"
                         if comb_reg else "SF + comb kernel (k_comb<3>: shared-memory form)",
                         launches_per_step=nwin,
                         launch_ms=comb_t / nwin, bytes_per_launch=comb_bytes / nwin,
                         kernel_ms_per_step=comb_t,
                         share_of_step=comb_t / ms_step, peak_source=pk["source"],
                         bytes_per_step=comb_bytes,
                         note="far below the HBM bound: instruction-issue and latency bound "
                              "(selection, window maxima, per-candidate medians)")
    dominant = roof_comb if roof_comb and roof_comb["kernel_ms_per_step"] > ndft_ms else roof_ndft
    metric = METRIC if (W, H) == (1280, 720) else METRIC.replace("1280x720", f"{W}x{H}")
    line = dict(
        metric=metric, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=ms_step, higher_is_better=True, scaling="weak",
        vs_baseline=None, dtype="f32", data="synthetic",
        config=dict(workload=WORKLOAD.format(W=W, H=H),
                    windows_per_step=nwin, events_per_step=events_step,
                    terms_per_step=terms_step, ms_per_window=ms_step / nwin,
                    stage_ms_per_step=dict(binning=statistics.mean(bin_ms), classify=f_avg,
                                           spectra=statistics.mean(spec_ms),
                                           comb=statistics.mean(comb_ms),
                                           labels_boxes=statistics.mean(box_ms)),
                    stage_note=("per-stage CUDA-event durations over 3 extra steps after the "
                                "timed region (a graph with event nodes, read back after each "
                                "step); " +
                                ("with the overlap tuning the comb of one window runs beside "
                                 "the binning and spectra of the next, so stages overlap in "
                                 "time and their sum exceeds the step"
                                 if int(tuning.get("overlap", 0)) else "stages in sequence")),
                    l2="inputs 8.3 GB per step, larger than L2; no flush",
                    tuning=dict(tuning, how=tune_note),
                    parallelism=f"replicas x{world}"),
        roofline=dominant,
        roofline_ndft=roof_ndft,
        roofline_comb=roof_comb,
        e2e=e2e,
        window_latency=lat,
        latency_sweep=sweep,
        labelled=labelled,
        peaks=dict(peaks, unit="per second, whole device",
                   how="ddhf_measure_pipes: 8 independent chains per thread, 8 blocks of "
                       "256 threads per SM, CUDA events"),
        softcomb=softc,
        spectrum_forms=forms,
        slide=slide,
        gpu_launches=int(graph_kernels) * args.steps,
        clocks=clk,
        plain=plain,
        cpu_baseline=cpu,
        stats=dict(n_rotor_last=st["n_rotor"], n_boxes_last=st["n_boxes"]),
    )
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
