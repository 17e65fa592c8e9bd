"""The no-allocation spectrum entry point against the context-based one.

ddhf_power_spectrum_noalloc serves callers that cannot allocate device
memory once they run (a real-time detector whose memory is reserved at
start-up, or a host program whose allocator owns the device). It runs the
same kernel as ddhf_power_spectrum(BLOCKED) with the default tuning, so its
spectra must be the same bits, on two calls in a row (its fixed scratch array
keeps the previous call's contents, so a stale counter would show up on the
second call), and once its first call has been made, later calls on any grid
must leave the device's free memory unchanged. This file is named to be
collected last.
"""
import numpy as np
import pytest
import torch

from paper_2603_08386_gb300 import build, ddhf, synth

pytestmark = pytest.mark.gpu


def _scene(seed, nb, step):
    s = synth.small_scene(seed, W=40, H=30, n_noise=40_000, drone_px=100,
                          grid=synth.hz_grid(0, step, nb))
    # one pixel with 3000 events goes through the whole-block (heavy) path
    rng = np.random.default_rng(seed)
    s.x = np.concatenate([s.x, np.full(3000, 5, np.int16)])
    s.y = np.concatenate([s.y, np.full(3000, 7, np.int16)])
    s.t = np.concatenate([s.t, rng.integers(0, s.window_us, 3000).astype(np.int64) + s.t0])
    s.p = np.concatenate([s.p, rng.choice(np.array([-1, 1], np.int8), 3000)])
    return s


def _reference(scene):
    """Per-pixel list and BLOCKED spectra from a context (default tuning)."""
    build.build()
    c = ddhf.Context(scene.W, scene.H, scene.grid, max_events=scene.n)
    x, y, t, p = ddhf.events_to_device(scene)
    c.bin_events(x, y, t, p, scene.t0, scene.window_us)
    csr = c.csr()
    ref = c.power_spectrum("blocked")
    c.stats()
    c.close()
    return csr, ref


def _call(scene, csr, P, flags):
    na = P.shape[0]
    ddhf.ddhf_power_spectrum_noalloc(ddhf.make_grid(*scene.grid), csr["offsets"], csr["ev"],
                                     csr["n_valid"], csr["active"], na, P, na, flags=flags)


def test_noalloc_equals_context_spectra_twice_without_allocating():
    # 750 bins runs 6 rows per lane, 333 bins 4 and 100 bins 1: the warm-up call
    # on the first grid must load the kernels of the others too
    cases = [_scene(3, 750, 2), _scene(4, 333, 10), _scene(5, 100, 10)]
    refs = [_reference(s) for s in cases]
    outs = [[torch.full(r.shape, -1.0, dtype=torch.float32, device="cuda") for _ in range(2)]
            for _, r in refs]
    flags = torch.full((len(cases), 2), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    _call(cases[0], refs[0][0], outs[0][0], flags[0, 0])  # first call in this context
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for i, (s, (csr, _)) in enumerate(zip(cases, refs)):
        for k in range(2):
            _call(s, csr, outs[i][k], flags[i, k])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    assert int(flags.abs().sum().item()) == 0, flags.tolist()
    for (_, ref), pair in zip(refs, outs):
        for P in pair:
            assert torch.equal(P, ref)


def test_noalloc_lists_out_of_order_give_the_same_rows():
    # a caller's active list need not follow the event array's order: shuffled,
    # with one pixel listed twice, the spectrum kernel streams such runs one
    # pixel at a time, and each row must be its pixel's row bit for bit
    s = _scene(6, 750, 2)
    csr, ref = _reference(s)
    act = csr["active"].long()
    na = act.numel()
    rng = np.random.default_rng(9)
    perm = torch.from_numpy(rng.permutation(na)).cuda()
    perm = torch.cat([perm, perm[:1]])  # a duplicate entry: overlapping ranges
    act2 = act[perm].to(torch.int32).contiguous()
    P = torch.full((perm.numel(), ref.shape[1]), -1.0, dtype=torch.float32, device="cuda")
    flags = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    ddhf.ddhf_power_spectrum_noalloc(ddhf.make_grid(*s.grid), csr["offsets"], csr["ev"],
                                     csr["n_valid"], act2, perm.numel(), P, perm.numel(),
                                     flags=flags)
    torch.cuda.synchronize()
    assert int(flags.item()) == 0
    assert torch.equal(P, ref[perm])


def test_noalloc_rejects_sizes_beyond_its_limit():
    build.build()
    g = ddhf.make_grid(0, 2000, synth.HZ_DENOM, 750)
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    P = torch.zeros((4, 750), dtype=torch.float32, device="cuda")
    with pytest.raises(ddhf.DDHFError) as e:
        ddhf.ddhf_power_spectrum_noalloc(g, dummy, dummy, (1 << 25) + 1, dummy, 4, P, 4)
    assert e.value.status == 1
    with pytest.raises(ddhf.DDHFError) as e:  # capacity below the active count
        ddhf.ddhf_power_spectrum_noalloc(g, dummy, dummy, 16, dummy, 4, P, 3)
    assert e.value.status == 1
