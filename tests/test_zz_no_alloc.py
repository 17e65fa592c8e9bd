"""The no-allocation spectrum entry point against the context-based one.

ddhf_power_spectrum_noalloc serves callers that cannot allocate device
memory once they run (a real-time detector whose memory is reserved at
start-up, or a host program whose allocator owns the device). It must give
the same spectra as ddhf_power_spectrum(BLOCKED) on the same per-pixel list,
on two calls in a row (its fixed scratch array keeps the previous call's
contents, so a stale counter would show up on the second call). This file is
named to be collected last.
"""
import numpy as np
import pytest
import torch

from paper_2603_08386_gb300 import build, ddhf, synth

pytestmark = pytest.mark.gpu

TOL_SPEC = 1e-4  # the spectrum tolerance of the parity tests: 1e-4 of each pixel's peak


def _case(scene):
    build.build()
    c = ddhf.Context(scene.W, scene.H, scene.grid, max_events=scene.n)
    x, y, t, p = ddhf.events_to_device(scene)
    c.bin_events(x, y, t, p, scene.t0, scene.window_us)
    csr = c.csr()
    ref = c.power_spectrum("blocked")
    c.stats()
    c.close()
    return csr, ref


def _close(P, ref):
    pk = ref.max(dim=1).values.clamp_min(1e-30)
    return float(((P - ref).abs().max(dim=1).values / pk).max().item())


@pytest.mark.parametrize("seed,nb,step", [(3, 750, 2), (4, 333, 10)])
def test_noalloc_matches_context_spectrum_twice(seed, nb, step):
    s = synth.small_scene(seed, W=40, H=30, n_noise=40_000, drone_px=100,
                          grid=synth.hz_grid(0, step, nb))
    # one pixel with 3000 events goes through the whole-block (heavy) path
    rng = np.random.default_rng(seed)
    s.x = np.concatenate([s.x, np.full(3000, 5, np.int16)])
    s.y = np.concatenate([s.y, np.full(3000, 7, np.int16)])
    s.t = np.concatenate([s.t, rng.integers(0, s.window_us, 3000).astype(np.int64) + s.t0])
    s.p = np.concatenate([s.p, rng.choice(np.array([-1, 1], np.int8), 3000)])
    csr, ref = _case(s)
    na = ref.shape[0]
    g = ddhf.make_grid(*s.grid)
    for _ in range(2):
        P = torch.full((na, nb), -1.0, dtype=torch.float32, device="cuda")
        ddhf.ddhf_power_spectrum_noalloc(g, csr["offsets"], csr["ev"], csr["n_valid"],
                                         csr["active"], na, P, na)
        torch.cuda.synchronize()
        assert _close(P, ref) <= TOL_SPEC


def test_noalloc_rejects_sizes_beyond_its_limit():
    build.build()
    g = ddhf.make_grid(0, 2000, synth.HZ_DENOM, 750)
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    P = torch.zeros((4, 750), dtype=torch.float32, device="cuda")
    with pytest.raises(ddhf.DDHFError) as e:
        ddhf.ddhf_power_spectrum_noalloc(g, dummy, dummy, (1 << 25) + 1, dummy, 4, P, 4)
    assert e.value.status == 1
