"""Soft comb score and its adjoint kernel (differentiation pattern) against
the FP64 oracle's analytic values, through the C ABI and the autograd wrapper.
Backgrounds B, f0 offsets, weights and widths come from the seeded generator."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_08386_gb300 import ddhf, synth

pytestmark = pytest.mark.gpu

TOL_S = 1e-4      # relative to the largest |S| of the batch
TOL_GRAD = 1e-3   # relative to the largest |gradient| of the batch (FP32 accumulation)


@pytest.fixture(scope="module")
def setup():
    from paper_2603_08386_gb300 import build
    build.build()
    s = synth.small_scene(71, W=48, H=40, n_noise=20_000, drone_px=160, f0_hz=150.0,
                          window_us=40_000, grid=synth.hz_grid(0, 2, 750))
    c = ddhf.Context(s.W, s.H, s.grid, max_events=s.n)
    x, y, t, p = ddhf.events_to_device(s)
    c.bin_events(x, y, t, p, s.t0, s.window_us)
    o = oracle.bin_events(s.W, s.H, s.x, s.y, s.t, s.p, s.t0, s.window_us)
    keys = np.array([k for k in s.drones[0]["keys"] if o["counts"][k] >= 6], np.int64)
    rng = np.random.default_rng(5)
    noise = rng.choice(np.flatnonzero(o["counts"] >= 6), 40, replace=False)
    keys = np.concatenate([keys, noise])
    n = keys.size
    f0 = (150.0 + rng.uniform(-2, 2, n)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, 6).astype(np.float32)
    sg = rng.uniform(1.0, 4.0, 6).astype(np.float32)
    B = rng.uniform(2.0, 20.0, n).astype(np.float32)
    g = rng.uniform(-1.0, 1.0, n).astype(np.float32)
    yield dict(s=s, c=c, o=o, keys=keys, f0=f0, w=w, sg=sg, B=B, g=g)
    c.close()


def oracle_all(d, Q, delta):
    o, out = d["o"], []
    for i, k in enumerate(d["keys"]):
        o0, o1 = o["offsets"][k], o["offsets"][k + 1]
        out.append(oracle.softcomb(o["tau"][o0:o1], o["pol"][o0:o1], float(d["f0"][i]),
                                   d["w"].astype(np.float64), d["sg"].astype(np.float64),
                                   delta, Q, float(d["B"][i]), tau_c=d["s"].window_us / 2))
    return out


@pytest.mark.parametrize("Q,delta", [(3, 2.0), (8, 0.5), (0, 2.0)])
def test_softcomb_forward_and_adjoint_match_oracle(setup, Q, delta):
    d = setup
    cu = lambda a, dt=torch.float32: torch.as_tensor(a, dtype=dt).cuda()
    pix = cu(d["keys"], torch.int32)
    f0, w, sg, B, g = cu(d["f0"]), cu(d["w"]), cu(d["sg"]), cu(d["B"]), cu(d["g"])
    n = d["keys"].size
    S = torch.empty(n, device="cuda")
    tc = d["s"].window_us / 2
    ddhf.ddhf_softcomb(d["c"].h, pix, f0, 6, Q, delta, tc, w, sg, B, S=S)
    gf0 = torch.empty(n, device="cuda")
    gw = torch.empty(6, device="cuda")
    gs = torch.empty(6, device="cuda")
    ddhf.ddhf_softcomb(d["c"].h, pix, f0, 6, Q, delta, tc, w, sg, B, grad_S=g, grad_f0=gf0,
                       grad_w=gw, grad_sigma=gs)
    ref = oracle_all(d, Q, delta)
    Sr = np.array([r["S"] for r in ref])
    np.testing.assert_allclose(S.cpu().numpy(), Sr, rtol=0, atol=TOL_S * np.abs(Sr).max())
    gf0r = d["g"] * np.array([r["dS_df0"] for r in ref])
    np.testing.assert_allclose(gf0.cpu().numpy(), gf0r, rtol=0,
                               atol=TOL_GRAD * np.abs(gf0r).max())
    gwr = (d["g"][:, None] * np.array([r["dS_dw"] for r in ref])).sum(0)
    np.testing.assert_allclose(gw.cpu().numpy(), gwr, rtol=0, atol=TOL_GRAD * np.abs(gwr).max())
    if Q > 0:
        gsr = (d["g"][:, None] * np.array([r["dS_dsigma"] for r in ref])).sum(0)
        np.testing.assert_allclose(gs.cpu().numpy(), gsr, rtol=0,
                                   atol=TOL_GRAD * np.abs(gsr).max())


def test_softcomb_autograd_and_refinement(setup):
    d = setup
    n = d["keys"].size
    pix = torch.as_tensor(d["keys"], dtype=torch.int32).cuda()
    B = torch.as_tensor(d["B"]).cuda()
    f0 = torch.as_tensor(d["f0"]).cuda().requires_grad_(True)
    w = torch.as_tensor(d["w"]).cuda().requires_grad_(True)
    sg = torch.as_tensor(d["sg"]).cuda().requires_grad_(True)
    tc = d["s"].window_us / 2
    S = ddhf.SoftComb.apply(f0, w, sg, d["c"].h, pix, B, 3, 2.0, tc)
    (S * torch.as_tensor(d["g"]).cuda()).sum().backward()
    ref = oracle_all(d, 3, 2.0)
    gwr = (d["g"][:, None] * np.array([r["dS_dw"] for r in ref])).sum(0)
    np.testing.assert_allclose(w.grad.cpu().numpy(), gwr, rtol=0, atol=TOL_GRAD * np.abs(gwr).max())
    # a few gradient-ascent steps on the drone pixels' f0 raise their soft score
    nd = int((np.isin(d["keys"], d["s"].drones[0]["keys"])).sum())
    f = torch.as_tensor(d["f0"][:nd]).cuda().requires_grad_(True)
    pd, Bd = pix[:nd].contiguous(), B[:nd].contiguous()
    wd, sd = torch.as_tensor(d["w"]).cuda(), torch.as_tensor(d["sg"]).cuda()
    s0 = ddhf.SoftComb.apply(f, wd, sd, d["c"].h, pd, Bd, 3, 2.0, tc).detach().clone()
    opt = torch.optim.SGD([f], lr=0.02)
    for _ in range(20):
        opt.zero_grad()
        (-ddhf.SoftComb.apply(f, wd, sd, d["c"].h, pd, Bd, 3, 2.0, tc).sum()).backward()
        torch.nn.utils.clip_grad_norm_([f], 50.0)
        opt.step()
    s1 = ddhf.SoftComb.apply(f, wd, sd, d["c"].h, pd, Bd, 3, 2.0, tc).detach()
    assert s1.sum() > s0.sum()


def test_spectrum_median_exact(setup):
    d = setup
    for N in (750, 333, 64):
        Pn = synth.synthetic_spectra(300, N, seed=N)
        c = ddhf.Context(10, 10, synth.hz_grid(0, 1, N), max_events=10)
        med = torch.empty(300, device="cuda")
        ddhf.ddhf_spectrum_median(c.h, torch.from_numpy(Pn).cuda(), 300, med)
        srt = np.sort(Pn, axis=1)
        if N % 2:
            ref = srt[:, (N - 1) // 2]
        else:
            ref = ((srt[:, N // 2 - 1] + srt[:, N // 2]) * np.float32(0.5)).astype(np.float32)
        np.testing.assert_array_equal(med.cpu().numpy(), ref)
        c.close()
