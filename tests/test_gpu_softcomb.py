"""Soft comb score and its adjoint kernel (differentiation pattern) against
the FP64 oracle's analytic values, through the C ABI and the autograd wrapper.
Backgrounds B, f0 offsets, weights and widths come from the seeded generator."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_08386_gb300 import ddhf, synth

pytestmark = pytest.mark.gpu

TOL_S = 1e-4      # of each pixel's own S (a sum of positive terms)
# FP32 accumulation of F and D over a pixel's events: each gradient element is
# compared against 1e-3 of its own condition scale, the sum of the absolute
# values of the terms it is made of, with dP/df = 2 Re(conj F D) bounded by
# 2 |F| |D| (the factors the FP32 sums produce); nothing is scaled by the
# batch's largest value.
TOL_GRAD = 1e-3


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
    """The oracle's S and analytic gradients per pixel, plus the condition
    scales of each output from its F and dF/df at the evaluation frequencies."""
    o, out = d["o"], []
    tc = d["s"].window_us / 2
    nh, nq = d["w"].size, 2 * Q + 1
    qd = np.arange(-Q, Q + 1) * delta
    w64, sg64 = d["w"].astype(np.float64), d["sg"].astype(np.float64)
    for i, k in enumerate(d["keys"]):
        o0, o1 = o["offsets"][k], o["offsets"][k + 1]
        tau, pol = o["tau"][o0:o1], o["pol"][o0:o1]
        r = oracle.softcomb(tau, pol, float(d["f0"][i]), w64, sg64, delta, Q, float(d["B"][i]),
                            tau_c=tc)
        fq = (np.arange(1, nh + 1)[:, None] * float(d["f0"][i]) + qd[None, :]).ravel()
        F, D = oracle.ndft_at(tau, pol, fq, tau_c=tc)
        F, D = F.reshape(nh, nq), D.reshape(nh, nq)
        G = np.exp(-(qd[None, :] ** 2) / (2.0 * sg64[:, None] ** 2))
        Z = G.sum(1, keepdims=True)
        Pw = np.abs(F) ** 2
        Bv = float(d["B"][i])
        fd_scale = np.abs(w64)[:, None] * (G / Z) * 2 * np.abs(F) * np.abs(D) / Bv  # [nh, nq]
        r["scale_df"] = fd_scale
        r["scale_df0"] = float((np.arange(1, nh + 1)[:, None] * fd_scale).sum())
        r["scale_S"] = float((np.abs(w64)[:, None] * (G / Z) * Pw).sum() / Bv)
        r["scale_dw"] = (G / Z * Pw).sum(1) / Bv
        A = (G / Z * Pw).sum(1)
        C = (G / Z * Pw * qd[None, :] ** 2).sum(1)
        E = (G / Z * qd[None, :] ** 2).sum(1)
        r["scale_dsigma"] = np.abs(w64) / (Bv * sg64 ** 3) * (C + A * E)
        out.append(r)
    return out


def worst(err, bar):
    """Largest error in units of its bar (<= 1 passes)."""
    return float(np.max(np.abs(err) / np.maximum(bar, 1e-30)))


@pytest.mark.parametrize("Q,delta", [(3, 2.0), (8, 0.5), (0, 2.0)])
def test_softcomb_forward_and_adjoint_match_oracle(setup, Q, delta):
    d = setup
    cu = lambda a, dt=torch.float32: torch.as_tensor(a, dtype=dt).cuda()
    pix = cu(d["keys"], torch.int32)
    f0, w, sg, B, g = cu(d["f0"]), cu(d["w"]), cu(d["sg"]), cu(d["B"]), cu(d["g"])
    n, nh, nq = d["keys"].size, 6, 2 * Q + 1
    S = torch.empty(n, device="cuda")
    tc = d["s"].window_us / 2
    ddhf.ddhf_softcomb(d["c"].h, pix, f0, nh, Q, delta, tc, w, sg, B, S=S)
    gf0 = torch.empty(n, device="cuda")
    gw = torch.empty(nh, device="cuda")
    gs = torch.empty(nh, device="cuda")
    gf = torch.full((n, nh, nq), float("nan"), device="cuda")
    ddhf.ddhf_softcomb(d["c"].h, pix, f0, nh, Q, delta, tc, w, sg, B, grad_S=g, grad_f0=gf0,
                       grad_w=gw, grad_sigma=gs, grad_f=gf)
    ref = oracle_all(d, Q, delta)
    gabs = np.abs(d["g"]).astype(np.float64)
    # S per pixel
    Sr = np.array([r["S"] for r in ref])
    assert worst(S.cpu().numpy() - Sr, TOL_S * np.array([r["scale_S"] for r in ref])) <= 1.0
    # dS/df0 per pixel
    gf0r = d["g"] * np.array([r["dS_df0"] for r in ref])
    bar0 = TOL_GRAD * gabs * np.array([r["scale_df0"] for r in ref])
    assert worst(gf0.cpu().numpy() - gf0r, bar0) <= 1.0
    # dS/df_hq per pixel, harmonic and evaluation frequency
    gfr = d["g"][:, None, None] * np.stack([r["dS_df"] for r in ref])
    barf = TOL_GRAD * gabs[:, None, None] * np.stack([r["scale_df"] for r in ref])
    gfg = gf.cpu().numpy()
    assert np.isfinite(gfg).all()
    assert worst(gfg - gfr, barf) <= 1.0
    # the per-frequency gradients sum to the fundamental's: dS/df0 = sum h dS/df_hq
    hsum = (np.arange(1, nh + 1)[None, :, None] * gfg).sum((1, 2))
    assert worst(hsum - gf0.cpu().numpy(), bar0) <= 1.0
    # dS/dw_h and dS/dsigma_h: signed sums over pixels, each against its own scale
    gwr = (d["g"][:, None] * np.array([r["dS_dw"] for r in ref])).sum(0)
    barw = TOL_GRAD * (gabs[:, None] * np.array([r["scale_dw"] for r in ref])).sum(0)
    assert worst(gw.cpu().numpy() - gwr, barw) <= 1.0
    if Q > 0:
        gsr = (d["g"][:, None] * np.array([r["dS_dsigma"] for r in ref])).sum(0)
        bars = TOL_GRAD * (gabs[:, None] * np.array([r["scale_dsigma"] for r in ref])).sum(0)
        assert worst(gs.cpu().numpy() - gsr, bars) <= 1.0


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
    barw = TOL_GRAD * (np.abs(d["g"])[:, None] * np.array([r["scale_dw"] for r in ref])).sum(0)
    assert worst(w.grad.cpu().numpy() - gwr, barw) <= 1.0
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


def test_stacked_batch_equals_single_windows(setup):
    # three windows laid out as one window of a sensor three times as tall
    # (ddhf.stack_windows, the C4 batch layout): one binning and one
    # ddhf_softcomb call per direction give every pixel the S and dS/df0 of its
    # own window's call, bit for bit
    scenes = [synth.small_scene(80 + b, W=48, H=40, n_noise=8_000, drone_px=60, f0_hz=150.0,
                                window_us=40_000, grid=synth.hz_grid(0, 2, 750)) for b in range(3)]
    W, H, grid, win = 48, 40, scenes[0].grid, scenes[0].window_us
    Q, delta, n_h = 3, 2.0, 6
    w = torch.linspace(0.5, 1.5, n_h, device="cuda")
    sg = torch.linspace(1.0, 3.0, n_h, device="cuda")
    per_S, per_g, per_keys = [], [], []
    for b, s in enumerate(scenes):
        c = ddhf.Context(W, H, grid, max_events=s.n)
        c.bin_events(*ddhf.events_to_device(s), s.t0, win)
        pix = c.csr()["active"].clone()
        keys = pix.long() + b * H * W
        f0 = 140.0 + (keys % 97).float().cuda() * 0.2
        B = 1.0 + (keys % 13).float().cuda()
        S = torch.empty(pix.numel(), device="cuda")
        ddhf.ddhf_softcomb(c.h, pix, f0, n_h, Q, delta, win / 2, w, sg, B, S=S)
        gf0 = torch.empty(pix.numel(), device="cuda")
        gw, gs = torch.empty(n_h, device="cuda"), torch.empty(n_h, device="cuda")
        ddhf.ddhf_softcomb(c.h, pix, f0, n_h, Q, delta, win / 2, w, sg, B,
                           grad_S=torch.ones_like(S), grad_f0=gf0, grad_w=gw, grad_sigma=gs)
        per_S.append(S)
        per_g.append(gf0)
        per_keys.append(keys)
        c.stats()
        c.close()
    xs, ys, ts, ps = ddhf.stack_windows([(s.x, s.y, s.t, s.p, s.t0) for s in scenes], H)
    cs = ddhf.Context(W, 3 * H, grid, max_events=xs.size)
    cs.bin_events(*(torch.from_numpy(a).cuda() for a in (xs, ys, ts, ps)), 0, win)
    pix = cs.csr()["active"].clone()
    keys = pix.long()
    assert torch.equal(keys, torch.cat(per_keys))
    f0 = 140.0 + (keys % 97).float().cuda() * 0.2
    B = 1.0 + (keys % 13).float().cuda()
    S = torch.empty(pix.numel(), device="cuda")
    ddhf.ddhf_softcomb(cs.h, pix, f0, n_h, Q, delta, win / 2, w, sg, B, S=S)
    gf0 = torch.empty(pix.numel(), device="cuda")
    gw, gs = torch.empty(n_h, device="cuda"), torch.empty(n_h, device="cuda")
    ddhf.ddhf_softcomb(cs.h, pix, f0, n_h, Q, delta, win / 2, w, sg, B,
                       grad_S=torch.ones_like(S), grad_f0=gf0, grad_w=gw, grad_sigma=gs)
    cs.stats()
    cs.close()
    assert torch.equal(S.view(torch.int32), torch.cat(per_S).view(torch.int32))
    assert torch.equal(gf0.view(torch.int32), torch.cat(per_g).view(torch.int32))
