"""Whole-window detection on labelled windows against the FP64 oracle.

The windows (synth.labelled_scene: the C3 noise recipe with two or three
drones) are scored with thresholds that separate the drones from the noise
(found on such windows; Table 2's own values flag the dense synthetic noise
too), so the detections are real boxes over a mask that is mostly empty.

Comparison, per active pixel, of the CUDA detector's rotor bit with the
oracle's (Eq. 6-11 in FP64 on the FP64 spectrum), wherever the oracle's
statistics are further from the thresholds than the arithmetic (1e-5) and
the FP32 spectrum can move them (oracle_margins states the bounds).
Boxes are compared without condition: always against the oracle's labelling
and Eq. 12 merging of the GPU's own mask, and against the oracle's boxes when
no pixel is inside its margin; each box's dominant frequency (its strongest
rotor pixel) against the oracle's selection on the GPU's own scores. The batched, graph-replayed call with the
benchmark's tuning (8 warps per block, overlapped windows, hybrid spectra for
pixels of at least 128 events) must give the same bits as one call per window.
"""
import numpy as np
import pytest
import torch

import oracle
import oracle_margins
from paper_2603_08386_gb300 import ddhf, synth

pytestmark = pytest.mark.gpu

BENCH_TUNING = dict(heavy_min=1024, warps_per_block=8, overlap=1, hybrid_min=128)
# thresholds inside Table 2's ranges that separate the labelled drones from
# the noise; Table 2's comb shape (M = 4, d = 3, h_min = 4: the register form
# of the fast comb) and a finer one (M = 8, d = 1: the shared-memory form)
CASES = [
    (400, dict(tau_sf=0.5, tau_comb=2.0, M=4, d=3, h_min=4, n_min=6, A_min=25, alpha=2.0)),
    (302, dict(tau_sf=0.5, tau_comb=3.0, M=8, d=1, h_min=3, n_min=4, A_min=25, alpha=2.0)),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2603_08386_gb300 import build
    build.build()
    oracle.build()
    ddhf.load()
    assert torch.cuda.is_available()
    yield


@pytest.mark.parametrize("seed,prm", CASES)
def test_labelled_detection_matches_oracle(seed, prm):
    s = synth.labelled_scene(seed, W=240, H=180, min_sep=100)
    params = ddhf.default_params(**prm)
    ev = ddhf.events_to_device(s)
    c = ddhf.Context(s.W, s.H, s.grid, params, max_events=s.n)
    c.set_tuning(**BENCH_TUNING)
    bx, nb, mask = c.detect(*ev, s.t0, s.window_us, cap=256, want_mask=True)
    sc = c.scores()
    f0b = torch.full((256,), -7, dtype=torch.int32, device="cuda")
    snrb = torch.zeros(256, device="cuda")
    medb = torch.full((256,), -3.0, device="cuda")
    ddhf.ddhf_box_frequencies(c.h, 0, bx, nb, 256, f0b, snrb, medb)
    P32 = c.power_spectrum("hybrid").cpu().numpy()  # the spectra the detection scored
    st = c.stats()
    c.close()
    n = int(nb.item())
    gmask = mask.cpu().numpy()
    act = sc["active"].cpu().numpy().astype(np.int64)
    # non-degenerate: real boxes over a mostly empty mask
    assert n >= 2 and st["n_active"] == act.size
    assert gmask.sum() < 0.2 * act.size
    # boxes are exactly the oracle's segmentation of the GPU's own mask
    ref_own = oracle_margins.segment(gmask, s.W, s.H, prm["A_min"], prm["alpha"], cap=256)
    np.testing.assert_array_equal(bx[:n].cpu().numpy(), ref_own)
    # each box's dominant bin: its strongest rotor pixel (Eq. 11 per pixel)
    rf, rs = oracle.box_frequencies(bx[:n].cpu().numpy(), act, gmask, sc["snr"].cpu().numpy(),
                                    sc["f0_bin"].cpu().numpy(), s.W)
    np.testing.assert_array_equal(f0b[:n].cpu().numpy(), rf)
    np.testing.assert_array_equal(snrb[:n].cpu().numpy().view(np.int32), rs.view(np.int32))
    assert (rf >= 0).all() and (f0b[n:].cpu().numpy() == -7).all()
    rm = oracle.box_median_hz(bx[:n].cpu().numpy(), act, gmask, sc["f0_bin"].cpu().numpy(), s.W,
                              s.grid)
    np.testing.assert_array_equal(medb[:n].cpu().numpy(), rm)
    # rotor bits against the FP64 oracle outside the margins
    b = oracle.bin_events(s.W, s.H, s.x, s.y, s.t, s.p, s.t0, s.window_us)
    np.testing.assert_array_equal(np.flatnonzero(b["counts"] >= prm["n_min"]), act)
    rot64, close = oracle_margins.decisions(b, act, P32, s.grid, prm)
    assert close.mean() < 0.01, close.sum()
    far = ~close
    np.testing.assert_array_equal(gmask[act[far]], rot64[far].astype(np.uint8))
    if not close.any():
        omask = np.zeros(s.W * s.H, np.uint8)
        omask[act[rot64]] = 1
        ref = oracle_margins.segment(omask, s.W, s.H, prm["A_min"], prm["alpha"], cap=256)
        np.testing.assert_array_equal(bx[:n].cpu().numpy(), ref)


def test_labelled_batch_graph_equals_single_windows():
    prm = CASES[0][1]
    params = ddhf.default_params(**prm)
    scenes = [synth.labelled_scene(sd, W=240, H=180, min_sep=100) for sd in (400, 302, 401)]
    W, H, grid = scenes[0].W, scenes[0].H, scenes[0].grid
    maxev = max(x.n for x in scenes)
    cap = 64
    single = []
    c1 = ddhf.Context(W, H, grid, params, max_events=maxev)
    c1.set_tuning(**BENCH_TUNING)
    for x in scenes:
        b1, n1, m1 = c1.detect(*ddhf.events_to_device(x), x.t0, x.window_us, cap=cap,
                               want_mask=True)
        single.append((b1[: int(n1.item())].clone(), m1.clone(), c1.scores()))
    c1.stats()
    c1.close()
    cb = ddhf.Context(W, H, grid, params, max_events=maxev, max_windows=len(scenes))
    cb.set_tuning(**BENCH_TUNING)
    dev = [ddhf.events_to_device(x) for x in scenes]
    wins = [(d[0], d[1], d[2], d[3], x.n, x.t0, x.window_us) for d, x in zip(dev, scenes)]
    boxes = torch.empty((len(scenes) * cap, 5), dtype=torch.int32, device="cuda")
    nbx = torch.zeros(len(scenes), dtype=torch.int32, device="cuda")
    masks = torch.empty((len(scenes), W * H), dtype=torch.uint8, device="cuda")
    for _ in range(3):  # capture, then replays
        boxes.fill_(-7)
        ddhf.ddhf_detect_batch(cb.h, wins, boxes, cap, nbx, masks, use_graph=True)
        torch.cuda.synchronize()
        for i, (bref, mref, sref) in enumerate(single):
            k = int(nbx[i].item())
            assert k >= 1
            assert torch.equal(boxes[i * cap: i * cap + k], bref)
            assert torch.equal(masks[i], mref)
            sb = cb.scores(slot=i)
            assert torch.equal(sb["snr"].view(torch.int32), sref["snr"].view(torch.int32))
            assert torch.equal(sb["f0_bin"], sref["f0_bin"])
    cb.stats()
    cb.close()
