"""Row-band sharding of the segmentation (Sec. 3.5, Eq. 12) on CPU: each
band's labels and components stand in for the device kernels' output (here
from the oracle's flood fill on the band's rows), the library's host merge
joins them, and the boxes must equal the oracle's on the whole mask. The
exchange step runs across two gloo ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2603_08386_gb300 import bands, ddhf


def band_part(mask, W, H, rows, b):
    """(edge labels [2, W] band-local, components [k, 6] in sensor coordinates)."""
    r0, r1 = rows[b], rows[b + 1]
    h = r1 - r0
    sub = np.ascontiguousarray(mask.reshape(H, W)[r0:r1])
    lab, _ = oracle.ccl8(sub.reshape(-1), W, h)
    lab2 = lab.reshape(h, W)
    comps = []
    for r in np.unique(lab[lab >= 0]):
        ys, xs = np.nonzero(lab2 == r)
        comps.append((int(r) + r0 * W, xs.min(), ys.min() + r0, xs.max(), ys.max() + r0, xs.size))
    c = np.array(comps, np.int32).reshape(-1, 6)
    return np.stack([lab2[0], lab2[h - 1]]).astype(np.int32), c


def crafted_mask(W, H, seed):
    """Random blobs plus shapes that cross band boundaries: vertical bars,
    diagonal chains (8- but not 4-connected across a row boundary) and
    U shapes whose arms meet only in another band."""
    rng = np.random.default_rng(seed)
    m = np.zeros((H, W), np.uint8)
    for _ in range(12):
        cx, cy = rng.integers(0, W), rng.integers(0, H)
        rx, ry = rng.integers(1, 5), rng.integers(1, 5)
        yy, xx = np.ogrid[:H, :W]
        m[((xx - cx) / rx) ** 2 + ((yy - cy) / ry) ** 2 <= 1.0] = 1
    for _ in range(3):
        x = rng.integers(0, W)
        y0 = rng.integers(0, H // 2)
        m[y0:y0 + rng.integers(H // 4, H // 2), x] = 1
    for _ in range(3):
        x, y = rng.integers(0, W - H // 2), rng.integers(0, H // 2)
        for k in range(H // 2):
            if 0 <= y + k < H and 0 <= x + k < W:
                m[y + k, x + k] = 1
    x = rng.integers(2, W - 8)
    m[H // 2 - 6:H // 2 + 1, x] = 1          # U: arms reach across row H/2 ...
    m[H // 2 - 6:H // 2 + 1, x + 5] = 1
    m[H // 2 - 6, x:x + 6] = 1                # ... and close above it
    m[rng.random((H, W)) < 0.02] = 1          # salt
    return m.reshape(-1)


@pytest.mark.parametrize("n_bands", [1, 2, 3, 5])
@pytest.mark.parametrize("A_min,alpha", [(1, 0.0), (4, 0.6), (9, 2.0), (147, 19.05)])
def test_merge_bands_equals_whole_sensor(n_bands, A_min, alpha):
    W, H = 48, 40
    params = ddhf.default_params(A_min=A_min, alpha=alpha)
    for seed in range(4):
        mask = crafted_mask(W, H, 100 + seed)
        rows = bands.band_rows(H, n_bands)
        parts = [band_part(mask, W, H, rows, b) for b in range(n_bands)]
        got, n = bands.exchange_and_merge(parts, rows, W, H, params)
        lab, _ = oracle.ccl8(mask, W, H)
        want = oracle.boxes(lab, W, H, A_min, alpha)
        assert n == want.shape[0]
        np.testing.assert_array_equal(got, want)


def test_merge_bands_capacity_and_invalid():
    W, H = 32, 24
    mask = crafted_mask(W, H, 7)
    rows = bands.band_rows(H, 2)
    parts = [band_part(mask, W, H, rows, b) for b in range(2)]
    params = ddhf.default_params(A_min=1, alpha=0.0)
    full, n = bands.exchange_and_merge(parts, rows, W, H, params)
    assert n >= 3
    few, n2 = bands.exchange_and_merge(parts, rows, W, H, params, cap=2)
    assert n2 == n and np.array_equal(few, full[:2])
    # an edge label with no component is rejected
    bad = [(parts[0][0].copy(), parts[0][1]), parts[1]]
    bad[0][0][1, :] = np.where(bad[0][0][1] >= 0, 10_000, -1)
    if (bad[0][0][1] >= 0).any():
        with pytest.raises(ddhf.DDHFError):
            bands.exchange_and_merge(bad, rows, W, H, params)
    with pytest.raises(ValueError):
        bands.band_rows(H, H + 1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    W, H = 48, 40
    mask = crafted_mask(W, H, 55)
    rows = bands.band_rows(H, world)
    params = ddhf.default_params(A_min=4, alpha=0.6)
    got, n = bands.exchange_and_merge(band_part(mask, W, H, rows, rank), rows, W, H, params)
    out.put((rank, got.tolist(), n))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_band_exchange():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    W, H = 48, 40
    lab, _ = oracle.ccl8(crafted_mask(W, H, 55), W, H)
    want = oracle.boxes(lab, W, H, 4, 0.6)
    for rank, got, n in res:
        assert n == want.shape[0]
        np.testing.assert_array_equal(np.array(got, np.int32).reshape(-1, 5), want)
