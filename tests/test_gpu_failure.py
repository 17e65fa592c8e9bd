"""Failure detection on the GPU without a GPU fault: the bounded union-find
loops of labelling and of the Eq. 12 merge are made to run out (the
context's loop limit lowered to 1), which must surface on the host as
DDHF_ERR_TIMEOUT with DDHF_FLAG_TIMEOUT set, after which the same context
(limit restored) labels the same mask exactly as the oracle does."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_08386_gb300 import ddhf, synth

pytestmark = pytest.mark.gpu

STATUS_TIMEOUT = 4
STATUS_CUDA = 2


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2603_08386_gb300 import build
    build.build()
    oracle.build()
    ddhf.load()
    assert torch.cuda.is_available()
    yield


def snake_mask(W, H):
    # rows 1, 3, 5, ... filled and joined at alternating ends: one 8-connected
    # component whose union-find paths are long
    m = np.zeros((H, W), np.uint8)
    for y in range(1, H - 1, 2):
        m[y, 1:W - 1] = 1
        if y + 2 < H - 1:
            m[y + 1, (W - 2) if (y // 2) % 2 == 0 else 1] = 1
    return m.reshape(-1)


def test_loop_limit_runs_out_and_context_recovers():
    W, H = 256, 40
    c = ddhf.Context(W, H, synth.hz_grid(0, 2, 750), max_events=16)
    m = snake_mask(W, H)
    mask = torch.from_numpy(m).cuda()
    ref, n_comp = oracle.ccl8(m, W, H)
    assert n_comp == 1
    bx = torch.empty((16, 5), dtype=torch.int32, device="cuda")
    nb = torch.zeros(1, dtype=torch.int32, device="cuda")

    ddhf.ddhf_set_loop_limit(c.h, 1)
    lab = c.label(mask)
    ddhf.ddhf_boxes(c.h, lab, bx, 16, nb)
    st = c.stats(raise_on_flags=False)
    assert st["status"] == STATUS_TIMEOUT
    assert st["device_flags"] & 2  # DDHF_FLAG_TIMEOUT
    # labels are unreliable after a run-out but stay in range
    got = lab.cpu().numpy()
    assert ((got == -1) | ((got >= 0) & (got < W * H))).all()

    # the flags were cleared by the read; with the default limit the same
    # context is exact again
    ddhf.ddhf_set_loop_limit(c.h, 1 << 24)
    lab = c.label(mask)
    ddhf.ddhf_boxes(c.h, lab, bx, 16, nb)
    st = c.stats(raise_on_flags=False)
    assert st["status"] == 0 and st["device_flags"] == 0
    np.testing.assert_array_equal(lab.cpu().numpy(), ref)
    assert int(nb.item()) == 1
    assert bx[0, :4].tolist() == [1, 1, W - 2, H - 2 - (H % 2 == 0)]
    with pytest.raises(ddhf.DDHFError):
        ddhf.ddhf_set_loop_limit(c.h, 0)
    c.close()


def test_injected_allocation_failure_releases_everything():
    # every allocation of ddhf_create fails in turn (a host-side injected
    # failure, no device fault): the call returns DDHF_ERR_CUDA, frees what it
    # had allocated, and a context made afterwards works
    s = synth.small_scene(9, W=40, H=30, n_noise=5_000)
    g = ddhf.make_grid(*s.grid)
    prm = ddhf.default_params()
    x, y, t, p = ddhf.events_to_device(s)
    warm = ddhf.Context(s.W, s.H, s.grid, max_events=s.n)  # loads the library's code first
    warm.detect(x, y, t, p, s.t0, s.window_us)
    warm.stats()
    warm.close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    failed = 0
    for n in range(0, 40, 3):
        ddhf.ddhf_debug_fail_alloc_after(n)
        try:
            h = ddhf.ddhf_create(s.W, s.H, g, prm, s.n, 2)
        except ddhf.DDHFError as e:
            assert e.status == 2
            failed += 1
            continue
        finally:
            ddhf.ddhf_debug_fail_alloc_after(-1)
        ddhf.ddhf_destroy(h)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert failed >= 5
    assert abs(free1 - free0) <= (2 << 20), (free0, free1)  # nothing leaked (2 MiB slack)
    c = ddhf.Context(s.W, s.H, s.grid, max_events=s.n)
    c.detect(x, y, t, p, s.t0, s.window_us)
    c.stats()
    c.close()


def test_guard_bytes_catch_a_write_outside_a_buffer():
    # a full detection leaves every workspace guard intact; one guard byte
    # overwritten from the host (inside the allocation: no stray device
    # access) is reported by the next ddhf_get_stats as an internal error
    s = synth.small_scene(31, W=64, H=48, n_noise=20_000, drone_px=120)
    c = ddhf.Context(s.W, s.H, s.grid, max_events=s.n, max_windows=2)
    x, y, t, p = ddhf.events_to_device(s)
    c.detect(x, y, t, p, s.t0, s.window_us, cap=64)
    st = c.stats()
    assert st["device_flags"] == 0
    for idx in (0, 7):
        ddhf.ddhf_debug_corrupt_guard(c.h, idx)
        st = c.stats(raise_on_flags=False)
        assert st["device_flags"] & 4 and st["status"] == STATUS_CUDA
    with pytest.raises(ddhf.DDHFError):
        ddhf.ddhf_debug_corrupt_guard(c.h, 1 << 20)
    c.close()


def test_out_of_range_keys_and_labels_are_skipped_and_reported():
    # caller-built device arrays with an index off the sensor: the kernels skip
    # the entry (no access outside the arrays) and ddhf_get_stats reports
    # DDHF_FLAG_INPUT as an invalid argument; the context stays usable
    s = synth.small_scene(32, W=40, H=30, n_noise=6_000, drone_px=60)
    c = ddhf.Context(s.W, s.H, s.grid, max_events=s.n)
    x, y, t, p = ddhf.events_to_device(s)
    c.bin_events(x, y, t, p, s.t0, s.window_us)
    pix = c.csr()["active"][:8].clone()
    pix[3] = s.W * s.H + 5
    n = pix.numel()
    ones = torch.ones(n, device="cuda")
    S = torch.full((n,), float("nan"), device="cuda")
    ddhf.ddhf_softcomb(c.h, pix, 150.0 * ones, 4, 2, 2.0, s.window_us / 2,
                       torch.ones(4, device="cuda"), torch.full((4,), 2.0, device="cuda"), ones, S=S)
    st = c.stats(raise_on_flags=False)
    assert st["device_flags"] & 8 and st["status"] == 1  # DDHF_ERR_INVALID_ARG
    assert float(S[3]) == 0.0 and torch.isfinite(S).all()
    lab = torch.full((s.W * s.H,), -1, dtype=torch.int32, device="cuda")
    lab[:4] = 0
    lab[10] = s.W * s.H + 100
    bx = torch.empty((16, 5), dtype=torch.int32, device="cuda")
    nb = torch.zeros(1, dtype=torch.int32, device="cuda")
    ddhf.ddhf_boxes(c.h, lab, bx, 16, nb)
    st = c.stats(raise_on_flags=False)
    assert st["device_flags"] & 8 and st["status"] == 1
    assert c.stats()["device_flags"] == 0  # reported once, then cleared
    c.close()
