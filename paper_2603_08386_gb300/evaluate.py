"""Detection quality on labelled synthetic windows and the Sec. 4.1
hyperparameter search, both driven through the CUDA detector.

Sec. 4.2 reports detections at 0.5 IoU against boxes that circumscribe a
drone's rotors; Sec. 4.1 tunes the thresholds of Sec. 3.4-3.5 by Bayesian
optimisation over the ranges of Table 2 (uniform priors, 50 random points,
then 300 expected-improvement steps) on a small labelled validation set.
The paper's recordings and labels are not available, so the windows here
are generated (synth.labelled_scene: the C3 noise recipe with 1-3 drones),
their ground truth is each drone's rotor bounding box, and the search runs
the detector of this library (ddhf_detect) at every evaluation.

Readings (the paper gives neither): boxes are inclusive pixel rectangles, so
a box (x0, y0, x1, y1) covers (x1 - x0 + 1)(y1 - y0 + 1) pixels; detections
are matched one to one, greedily in decreasing IoU (ties by prediction,
then ground-truth index), and a pair counts when IoU >= 0.5; F1 =
2 TP / (2 TP + FP + FN) over all windows of a set (1 when the set has
neither detections nor drones).

  python -m paper_2603_08386_gb300.evaluate [--n-init 50] [--n-iter 300]
prints one JSON line: Table 2's F1 and the tuned parameters' F1 on the
validation and held-out windows.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import bo, synth

# Table 2: (name, lower, upper, integer) of the search space
TABLE2_SPACE = [("tau_sf", 0.3, 0.98, False), ("tau_comb", 1.5, 6.0, False),
                ("M", 4, 16, True), ("d", 0, 4, True), ("h_min", 2, 8, True),
                ("n_min", 2, 10, True), ("A_min", 9, 196, True), ("alpha", 3.0, 20.0, False)]


def box_iou(a, b) -> float:
    """IoU of two inclusive pixel boxes (x0, y0, x1, y1)."""
    iw = min(a[2], b[2]) - max(a[0], b[0]) + 1
    ih = min(a[3], b[3]) - max(a[1], b[1]) + 1
    inter = max(iw, 0) * max(ih, 0)
    area_a = (a[2] - a[0] + 1) * (a[3] - a[1] + 1)
    area_b = (b[2] - b[0] + 1) * (b[3] - b[1] + 1)
    return inter / float(area_a + area_b - inter)


def match(pred, gt, thr=0.5):
    """(TP, FP, FN) of one window: one-to-one greedy matching by IoU."""
    pairs = []
    for i, p in enumerate(pred):
        for j, g in enumerate(gt):
            v = box_iou(p, g)
            if v >= thr:
                pairs.append((-v, i, j))
    pairs.sort()
    used_p, used_g = set(), set()
    for _, i, j in pairs:
        if i not in used_p and j not in used_g:
            used_p.add(i)
            used_g.add(j)
    tp = len(used_p)
    return tp, len(pred) - tp, len(gt) - tp


def f1_score(tp, fp, fn) -> float:
    den = 2 * tp + fp + fn
    return 1.0 if den == 0 else 2.0 * tp / den


def gt_boxes(scene):
    return [tuple(d["box"]) for d in scene.drones if d["box"] is not None]


class Evaluator:
    """F1 at an IoU threshold of a parameter set over windows of one sensor
    size, each detected by ddhf_detect on the current CUDA device."""

    def __init__(self, scenes, thr=0.5, cap=256):
        import torch

        from . import ddhf
        self.torch, self.ddhf = torch, ddhf
        s0 = scenes[0]
        assert all((s.W, s.H, tuple(s.grid)) == (s0.W, s0.H, tuple(s0.grid)) for s in scenes)
        self.ctx = ddhf.Context(s0.W, s0.H, s0.grid, max_events=max(s.n for s in scenes))
        self.wins = [(ddhf.events_to_device(s), s.t0, s.window_us) for s in scenes]
        self.gt = [gt_boxes(s) for s in scenes]
        self.thr, self.cap = thr, cap

    def counts(self, params):
        self.ctx.set_params(params)
        tp = fp = fn = 0
        for (ev, t0, wus), gt in zip(self.wins, self.gt):
            bx, nb, _ = self.ctx.detect(*ev, t0, wus, cap=self.cap)
            n = int(nb.item())
            pred = [tuple(b[:4]) for b in bx[: min(n, self.cap)].cpu().numpy().tolist()]
            a, b, c = match(pred, gt, self.thr)
            tp, fp, fn = tp + a, fp + b + max(n - self.cap, 0), fn + c
        self.ctx.stats()
        return tp, fp, fn

    def f1(self, params) -> float:
        return f1_score(*self.counts(params))

    def close(self):
        self.ctx.close()


def params_of(vals: dict):
    from . import ddhf
    return ddhf.default_params(**vals)


def tune(evaluator, n_init=50, n_iter=300, seed=0, log=None):
    """Sec. 4.1's search over Table 2's ranges, maximising the evaluator's F1."""
    space = bo.Space(TABLE2_SPACE)
    return bo.maximise(lambda v: evaluator.f1(params_of(v)), space, n_init=n_init,
                       n_iter=n_iter, seed=seed, log=log)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-init", type=int, default=50)
    ap.add_argument("--n-iter", type=int, default=300)
    ap.add_argument("--val", type=int, default=4, help="validation windows (320x240)")
    ap.add_argument("--test", type=int, default=8, help="held-out windows (320x240)")
    ap.add_argument("--c3", type=int, default=2, help="held-out 1280x720 C3 windows")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    import torch
    from . import build, ddhf
    build.build()
    torch.cuda.set_device(0)
    t_start = time.time()
    val = Evaluator([synth.labelled_scene(100 + i) for i in range(args.val)])
    test = Evaluator([synth.labelled_scene(200 + i) for i in range(args.test)])
    table2 = {k: getattr(ddhf.default_params(), k) for k, *_ in TABLE2_SPACE}
    best, best_f1, hist = tune(val, args.n_init, args.n_iter, args.seed)
    out = dict(
        search=dict(space="Table 2 ranges", n_init=args.n_init, n_iter=args.n_iter,
                    evaluations=len(hist), validation_windows=args.val, seed=args.seed),
        table2=dict(params=table2, val_f1=val.f1(params_of(table2)),
                    test_f1=test.f1(params_of(table2))),
        tuned=dict(params=best, val_f1=best_f1, test_f1=test.f1(params_of(best))),
        test_windows=args.test, iou=0.5)
    val.close()
    test.close()
    if args.c3:
        c3 = Evaluator([synth.config3_window(0, w) for w in range(args.c3)])
        out["c3"] = dict(windows=args.c3, table2_f1=c3.f1(params_of(table2)),
                         tuned_f1=c3.f1(params_of(best)),
                         tuned_counts=c3.counts(params_of(best)))
        c3.close()
    out["seconds"] = time.time() - t_start
    print(json.dumps(out))


if __name__ == "__main__":
    main()
