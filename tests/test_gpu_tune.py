"""Autotuner of the batched detection: picks a launchable candidate, caches
it, reuses the cache, and the tuned kernel keeps the parity properties."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2603_08386_gb300 import ddhf, synth, tune

pytestmark = pytest.mark.gpu


def test_autotune_choice_cache_and_parity(tmp_path):
    from paper_2603_08386_gb300 import build
    build.build()
    scenes = [synth.small_scene(90 + i, W=64, H=48, n_noise=40_000, drone_px=150,
                                grid=synth.hz_grid(0, 2, 750)) for i in range(3)]
    W, H, cap = 64, 48, 64
    maxev = max(s.n for s in scenes)
    c = ddhf.Context(W, H, scenes[0].grid, max_events=maxev, max_windows=len(scenes))
    dev = [ddhf.events_to_device(s) for s in scenes]
    wins = [(d[0], d[1], d[2], d[3], s.n, s.t0, s.window_us) for d, s in zip(dev, scenes)]
    boxes = torch.empty((len(scenes) * cap, 5), dtype=torch.int32, device="cuda")
    nb = torch.zeros(len(scenes), dtype=torch.int32, device="cuda")
    cache = str(tmp_path / "tune.json")
    cands = [dict(heavy_min=64, warps_per_block=4, blocks_per_sm=0, rows_per_lane=0),
             dict(heavy_min=1024, warps_per_block=8, blocks_per_sm=0, rows_per_lane=4),
             dict(heavy_min=256, warps_per_block=2, blocks_per_sm=1, rows_per_lane=8),
             dict(heavy_min=512, warps_per_block=4, blocks_per_sm=0, rows_per_lane=0, fuse=0,
                  overlap=1)]
    best, timings = tune.autotune(c, wins, boxes, cap, nb, candidates=cands, cache_path=cache)
    assert best in cands and len(timings) == len(cands)
    assert min(timings.values()) == timings[json.dumps(best, sort_keys=True)]
    cur = ddhf.ddhf_get_tuning(c.h)
    assert all(cur[k] == v for k, v in best.items())
    assert os.path.exists(cache)
    again, _ = tune.autotune(c, wins, boxes, cap, nb, candidates=cands[:1], cache_path=cache)
    assert again == best  # served from the cache, no new timing
    c.close()
    # under each candidate: spectra within tolerance of the oracle, fused == unfused
    s = scenes[0]
    o = oracle.bin_events(s.W, s.H, s.x, s.y, s.t, s.p, s.t0, s.window_us)
    for cand in cands:
        c1 = ddhf.Context(W, H, s.grid, max_events=s.n)
        c1.set_tuning(**cand)
        x, y, t, p = dev[0]
        _, _, mask = c1.detect(x, y, t, p, s.t0, s.window_us, want_mask=True)
        sc = c1.scores()
        P = c1.power_spectrum("blocked")
        out = c1.comb_score(P)
        assert torch.equal(out["mask"], mask) and torch.equal(out["f0_bin"], sc["f0_bin"])
        act = sc["active"].cpu().numpy()
        Pn = P.cpu().numpy()
        for a in range(0, len(act), 17):
            k = act[a]
            ref = oracle.ndft(o["tau"][o["offsets"][k]:o["offsets"][k + 1]],
                              o["pol"][o["offsets"][k]:o["offsets"][k + 1]], *s.grid)
            assert np.abs(Pn[a] - ref).max() <= 1e-4 * ref.max()
        c1.stats()
        c1.close()
