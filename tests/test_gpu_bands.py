"""Row bands on the GPU: each band's context (row offset) bins only its rows,
its rotor mask equals the whole sensor's rows bit for bit, and the merged
boxes equal ddhf_detect's on the whole sensor. The bands run one after the
other on one GPU; across GPUs each rank runs one band and the exchange is
the all-gather tested on CPU."""
import numpy as np
import pytest
import torch

from paper_2603_08386_gb300 import bands, ddhf, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_bands", [2, 3])
@pytest.mark.parametrize("prm", [dict(), dict(A_min=4, alpha=0.6)])
def test_bands_equal_whole_sensor(n_bands, prm):
    s = synth.small_scene(71, W=64, H=48, n_noise=50_000, drone_px=200,
                          grid=synth.hz_grid(0, 2, 750))
    params = ddhf.default_params(**prm)
    x, y, t, p = ddhf.events_to_device(s)
    c = ddhf.Context(s.W, s.H, s.grid, params, max_events=s.n)
    cap = 256
    bx = torch.empty((cap, 5), dtype=torch.int32, device="cuda")
    nb = torch.zeros(1, dtype=torch.int32, device="cuda")
    mask = torch.empty(s.W * s.H, dtype=torch.uint8, device="cuda")
    ddhf.ddhf_detect(c.h, x, y, t, p, s.n, s.t0, s.window_us, bx, cap, nb, mask)
    st = c.stats()
    c.close()
    want = bx[: int(nb.item())].cpu().numpy()
    full_mask = mask.cpu().numpy().reshape(s.H, s.W)
    assert full_mask.any()

    parts, valid, masks = [], 0, []
    for b in range(n_bands):
        bd = bands.BandDetector(s.W, s.H, s.grid, b, n_bands, params, max_events=s.n)
        parts.append(bd.part(x, y, t, p, s.t0, s.window_us))
        masks.append(bd.mask.cpu().numpy().reshape(bd.h, s.W))
        valid += bd.ctx.stats()["n_valid"]
        bd.close()
    assert valid == st["n_valid"]
    np.testing.assert_array_equal(np.concatenate(masks), full_mask)
    got, n = bands.exchange_and_merge(parts, bands.band_rows(s.H, n_bands), s.W, s.H, params, cap)
    assert n == want.shape[0]
    np.testing.assert_array_equal(got, want)
