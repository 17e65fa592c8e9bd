"""Hybrid spectra (DDHF_FORM_HYBRID and the hybrid_min tuning) through the C
ABI against the FP64 oracle's Eq. 6.

Pixels with many events go through the uniform-grid route the footnote to
Sec. 3.3 mentions (spreading with an exponential-of-semicircle kernel, one
dense product with a shared table, deconvolution); the others through the
blocked kernel, whose rows must stay bit-identical to DDHF_FORM_BLOCKED.
Bar: every pixel within 1e-4 of its peak power, as for the other forms.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_08386_gb300 import ddhf, synth

pytestmark = pytest.mark.gpu

TOL_SPEC = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2603_08386_gb300 import build
    build.build()
    oracle.build()
    ddhf.load()
    assert torch.cuda.is_available()
    yield


def plan(grid, window_us, hybrid_min):
    """Threshold and grid rows of the hybrid route (the rule ddhf.h states)."""
    a0, da, D, N = grid
    s = D // (2 * da * N)
    if s < 1:
        return None
    G = (window_us - 1) // s + 8
    if G < 16 or G > 1024:
        return None
    return max(hybrid_min, 16, -(-G // 2)), G


def spectra(scene, form, **tuning):
    c = ddhf.Context(scene.W, scene.H, scene.grid, max_events=scene.n)
    if tuning:
        c.set_tuning(**tuning)
    x, y, t, p = ddhf.events_to_device(scene)
    c.bin_events(x, y, t, p, scene.t0, scene.window_us)
    P = c.power_spectrum(form).cpu().numpy()
    act = c.csr()["active"].cpu().numpy()
    c.stats()
    c.close()
    return P, act


def check_rows(scene, P, act, rows):
    o = oracle.bin_events(scene.W, scene.H, scene.x, scene.y, scene.t, scene.p, scene.t0,
                          scene.window_us)
    worst = 0.0
    for a in rows:
        k = act[a]
        o0, o1 = o["offsets"][k], o["offsets"][k + 1]
        ref = oracle.ndft(o["tau"][o0:o1], o["pol"][o0:o1], *scene.grid)
        err = np.abs(P[a].astype(np.float64) - ref).max() / ref.max()
        worst = max(worst, err)
        assert err <= TOL_SPEC, (a, o1 - o0, err)
    return o, worst


GRIDS = {
    # C3's grid: s = 333 us, G = 98 over 30 ms
    "c3": dict(grid=synth.hz_grid(0, 2, 750), window_us=30_000),
    # C2's grid over 50 ms: s = 250 us, G = 208
    "c2": dict(grid=synth.hz_grid(0, 1, 2000), window_us=50_000),
    # C1's grid over 20 ms: s = 500 us, G = 47
    "c1": dict(grid=synth.hz_grid(0, 10, 100), window_us=20_000),
    # a band away from 0 Hz (centre phase of the events not trivial)
    "band": dict(grid=synth.hz_grid(97.5, 1.5, 600), window_us=30_000),
    # the paper's normalised modes k = 0..99 over a 20 ms window: s = 100, G = 207
    "modes": dict(grid=synth.mode_grid(20_000, 100), window_us=20_000),
}


@pytest.mark.parametrize("name", list(GRIDS))
def test_hybrid_matches_oracle_and_blocked_rows(name):
    cfg = GRIDS[name]
    s = synth.config3_window(stream=0, window=1, seed=77, W=120, H=96,
                             window_us=cfg["window_us"], mean_per_px=30.0, grid=cfg["grid"])
    thr, G = plan(s.grid, s.window_us, 32)
    P_h, act = spectra(s, "hybrid", hybrid_min=32)
    P_b, act_b = spectra(s, "blocked")
    np.testing.assert_array_equal(act, act_b)
    o = oracle.bin_events(s.W, s.H, s.x, s.y, s.t, s.p, s.t0, s.window_us)
    counts = o["counts"][act]
    heavy = np.flatnonzero(counts >= thr)
    light = np.flatnonzero(counts < thr)
    assert len(heavy) >= 50, (thr, G, len(heavy))
    # light rows: the same blocked kernel, bit for bit
    np.testing.assert_array_equal(P_h[light].view(np.uint32), P_b[light].view(np.uint32))
    # grid rows: the heaviest, a ragged spread of the rest, the ones at the threshold
    rng = np.random.default_rng(5)
    by_count = heavy[np.argsort(-counts[heavy], kind="stable")]
    rows = np.unique(np.concatenate([by_count[:6], rng.choice(heavy, min(120, len(heavy)),
                                                              replace=False),
                                     heavy[counts[heavy] == counts[heavy].min()][:10]]))
    _, worst = check_rows(s, P_h, act, rows)
    print(f"{name}: thr {thr}, G {G}, {len(heavy)} grid pixels, worst {worst:.2e}")


def test_hybrid_drone_pixels_and_periodic_peaks():
    # rotor pixels of a drone through the grid route keep their comb peaks
    s = synth.small_scene(11, W=64, H=48, n_noise=120_000, drone_px=300,
                          grid=synth.hz_grid(0, 2, 750))
    P_h, act = spectra(s, "hybrid", hybrid_min=16)
    o = oracle.bin_events(s.W, s.H, s.x, s.y, s.t, s.p, s.t0, s.window_us)
    thr, _ = plan(s.grid, s.window_us, 16)
    counts = o["counts"][act]
    rows = np.flatnonzero(counts >= thr)[:150]
    assert len(rows) >= 20
    check_rows(s, P_h, act, rows)


def test_hybrid_long_window_runs_blocked():
    # 400 ms at C3's grid needs G = 1209 > 1024 grid rows: every pixel takes
    # the blocked kernel, so the result is the BLOCKED form's bit for bit
    s = synth.config3_window(stream=0, window=0, seed=78, W=48, H=40, window_us=400_000,
                             mean_per_px=40.0)
    assert plan(s.grid, s.window_us, 32) is None
    P_h, _ = spectra(s, "hybrid", hybrid_min=32)
    P_b, _ = spectra(s, "blocked")
    np.testing.assert_array_equal(P_h.view(np.uint32), P_b.view(np.uint32))


def test_hybrid_empty_and_no_heavy_pixels():
    s = synth.small_scene(12, W=40, H=30, n_noise=3000, drone_px=20,
                          grid=synth.hz_grid(0, 2, 750))
    P_h, act = spectra(s, "hybrid", hybrid_min=10_000)
    P_b, _ = spectra(s, "blocked")
    np.testing.assert_array_equal(P_h.view(np.uint32), P_b.view(np.uint32))
    # a window with no events at all
    for f in ("x", "y", "t", "p"):
        setattr(s, f, getattr(s, f)[:0])
    c = ddhf.Context(s.W, s.H, s.grid, max_events=16)
    c.set_tuning(hybrid_min=32)
    x, y, t, p = ddhf.events_to_device(s)
    c.bin_events(x, y, t, p, s.t0, s.window_us)
    assert c.power_spectrum("hybrid").shape[0] == 0
    c.stats()
    c.close()


def test_detect_with_hybrid_tuning():
    # ddhf_detect (unfused) with hybrid_min set scores the same spectra that
    # DDHF_FORM_HYBRID returns: the comb on those gives the same mask, bit for
    # bit, and the batched call (direct and as a replayed graph) repeats it
    s = synth.small_scene(14, W=64, H=48, n_noise=150_000, drone_px=300,
                          grid=synth.hz_grid(0, 2, 750))
    c = ddhf.Context(s.W, s.H, s.grid, max_events=s.n, max_windows=2)
    c.set_tuning(hybrid_min=24, fuse=0)
    ev = ddhf.events_to_device(s)
    bx, nb, mask = c.detect(*ev, s.t0, s.window_us, want_mask=True)
    n = int(nb.item())
    assert n >= 1
    c.bin_events(*ev, s.t0, s.window_us)
    P = c.power_spectrum("hybrid")
    assert torch.equal(c.comb_score(P)["mask"], mask)
    cap = 64
    wins = [(*ev, s.n, s.t0, s.window_us)] * 2
    boxes = torch.empty((2 * cap, 5), dtype=torch.int32, device="cuda")
    nbx = torch.zeros(2, dtype=torch.int32, device="cuda")
    masks = torch.empty((2, s.W * s.H), dtype=torch.uint8, device="cuda")
    for overlap, use_graph in ((0, False), (0, True), (0, True), (1, True), (1, True)):
        c.set_tuning(overlap=overlap)
        boxes.fill_(-7)
        masks.fill_(3)
        ddhf.ddhf_detect_batch(c.h, wins, boxes, cap, nbx, masks, use_graph=use_graph)
        torch.cuda.synchronize()
        for w in range(2):
            assert int(nbx[w].item()) == n
            assert torch.equal(boxes[w * cap: w * cap + n], bx[:n])
            assert torch.equal(masks[w], mask)
    c.stats()
    c.close()


def test_c3_window_full_size_hybrid_sampled():
    s = synth.config3_window(stream=2, window=5)
    thr, G = plan(s.grid, s.window_us, 64)
    P_h, act = spectra(s, "hybrid", hybrid_min=64)
    o = oracle.bin_events(s.W, s.H, s.x, s.y, s.t, s.p, s.t0, s.window_us)
    counts = o["counts"][act]
    heavy = np.flatnonzero(counts >= thr)
    rng = np.random.default_rng(9)
    rows = np.unique(np.concatenate([heavy[np.argsort(-counts[heavy], kind="stable")[:4]],
                                     rng.choice(heavy, 60, replace=False),
                                     rng.choice(np.flatnonzero(counts < thr), 40,
                                                replace=False)]))
    _, worst = check_rows(s, P_h, act, rows)
    print(f"C3 full window: thr {thr}, G {G}, {len(heavy)} grid pixels of {len(act)}, "
          f"worst {worst:.2e}")
