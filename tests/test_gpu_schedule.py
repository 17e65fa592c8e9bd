"""How the work is spread over the GPU does not change the results.

The blocked NDFT kernel streams the light pixels in runs whose length follows
the number of active pixels per warp of its grid (16 pixels on a dense
window, down to one on a sparse one), and the comb kernel takes its pixels
from a counter. A pixel's events are accumulated in the same order whatever
run it falls in, so the spectra must be the same bits for grids of different
sizes (which choose different run lengths), and the comb's outputs the same
bits on repeated calls.
"""
import pytest
import torch

from paper_2603_08386_gb300 import build, ddhf, synth

pytestmark = pytest.mark.gpu

# (warps per block, blocks per SM): 2432, 608 and 304 warps on 152 SMs, so the
# run length differs between them at every density below
GRIDS = [dict(), dict(blocks_per_sm=1), dict(warps_per_block=2, blocks_per_sm=1)]


def _spectra(scene, x, y, t, p, **tuning):
    c = ddhf.Context(scene.W, scene.H, scene.grid, max_events=scene.n)
    # every pixel through the light (run-streamed) path: no block-per-pixel
    # heavy path and no hybrid grid route
    c.set_tuning(heavy_min=1 << 30, hybrid_min=0, **tuning)
    c.bin_events(x, y, t, p, scene.t0, scene.window_us)
    P = c.power_spectrum("blocked").clone()
    c.stats()
    c.close()
    return P


@pytest.mark.parametrize("mean", [1.0, 4.0, 21.7])
def test_blocked_spectra_do_not_depend_on_the_grid(mean):
    build.build()
    s = synth.config3_window(0, 0, seed=1003, W=640, H=360, mean_per_px=mean)
    x, y, t, p = ddhf.events_to_device(s)
    outs = [_spectra(s, x, y, t, p, **g) for g in GRIDS]
    assert outs[0].shape[0] > 1000
    for P in outs[1:]:
        assert P.shape == outs[0].shape
        assert torch.equal(P, outs[0])


def test_comb_scores_repeat_bit_for_bit():
    build.build()
    s = synth.config3_window(0, 0, seed=1004, W=640, H=360, mean_per_px=6.0)
    x, y, t, p = ddhf.events_to_device(s)
    c = ddhf.Context(s.W, s.H, s.grid, max_events=s.n)
    c.bin_events(x, y, t, p, s.t0, s.window_us)
    P = c.power_spectrum("blocked")
    first = {k: v.clone() for k, v in c.comb_score(P).items()}
    assert first["snr"].numel() > 1000
    for _ in range(3):
        again = c.comb_score(P)
        for k, v in first.items():
            assert torch.equal(again[k], v), k
    c.stats()
    c.close()
