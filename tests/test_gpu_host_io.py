"""Host-input batch detection: events in page-locked host memory, copies of
the next group of windows overlapped with the current one; boxes, counts and
masks must equal the device-input path exactly, for more windows than the
context's window slots, with one and with three slots (groups of 3 and 2) and
with the fused, unfused and overlapped tunings."""
import numpy as np
import pytest
import torch

from paper_2603_08386_gb300 import ddhf, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fuse,max_windows,overlap", [(0, 1, 0), (1, 1, 0), (0, 3, 1), (1, 3, 0)])
def test_host_batch_equals_device_path(fuse, max_windows, overlap):
    # with 3 window slots the 5 windows go through as groups of 3 and 2 by the
    # batched detection (the overlapped form with overlap 1)
    scenes = [synth.small_scene(80 + i, W=48, H=40, n_noise=15_000 + 4000 * i, drone_px=120,
                                grid=synth.hz_grid(0, 2, 750)) for i in range(5)]
    W, H, cap = 48, 40, 64
    maxev = max(sc.n for sc in scenes)
    c = ddhf.Context(W, H, scenes[0].grid, max_events=maxev, max_windows=max_windows)
    c.set_tuning(fuse=fuse, overlap=overlap)
    want = []
    bx = torch.empty((cap, 5), dtype=torch.int32, device="cuda")
    nb = torch.zeros(1, dtype=torch.int32, device="cuda")
    m = torch.empty(W * H, dtype=torch.uint8, device="cuda")
    for sc in scenes:
        x, y, t, p = ddhf.events_to_device(sc)
        ddhf.ddhf_detect(c.h, x, y, t, p, sc.n, sc.t0, sc.window_us, bx, cap, nb, m)
        n = int(nb.item())
        want.append((bx[:min(n, cap)].cpu().numpy(), n, m.cpu().numpy()))
    host = [tuple(torch.from_numpy(a).pin_memory() for a in (sc.x, sc.y, sc.t, sc.p))
            for sc in scenes]
    wins = [(h[0], h[1], h[2], h[3], sc.n, sc.t0, sc.window_us) for h, sc in zip(host, scenes)]
    hb = torch.full((len(scenes) * cap, 5), -3, dtype=torch.int32).pin_memory()
    hn = torch.zeros(len(scenes), dtype=torch.int32).pin_memory()
    hm = torch.zeros((len(scenes), W * H), dtype=torch.uint8).pin_memory()
    for _ in range(2):  # twice: the staging buffers and events are reused
        ddhf.ddhf_detect_batch_host(c.h, wins, hb, cap, hn, hm)
        torch.cuda.synchronize()
        for i, (wb, wn, wm) in enumerate(want):
            assert int(hn[i]) == wn
            np.testing.assert_array_equal(hb[i * cap: i * cap + min(wn, cap)].numpy(), wb)
            np.testing.assert_array_equal(hm[i].numpy(), wm)
    c.stats()
    c.close()


def test_host_batch_rejects_bad_arguments():
    sc = synth.small_scene(90, W=32, H=24, n_noise=2000, drone_px=40)
    c = ddhf.Context(32, 24, sc.grid, max_events=sc.n)
    h = tuple(torch.from_numpy(a) for a in (sc.x, sc.y, sc.t, sc.p))
    hb = torch.zeros((8, 5), dtype=torch.int32)
    hn = torch.zeros(1, dtype=torch.int32)
    with pytest.raises(ddhf.DDHFError):  # more events than max_events
        ddhf.ddhf_detect_batch_host(c.h, [(h[0], h[1], h[2], h[3], sc.n + 1, 0, sc.window_us)],
                                    hb, 8, hn)
    with pytest.raises(ddhf.DDHFError):  # bad window length
        ddhf.ddhf_detect_batch_host(c.h, [(h[0], h[1], h[2], h[3], sc.n, 0, 0)], hb, 8, hn)
    c.close()
