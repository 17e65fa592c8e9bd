"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formula: each checks it against a
library routine (numpy stable sort, FFT, scipy labelling), a closed form, an
invariant, or an exhaustive brute force on tiny inputs, so that a dropped
term, a wrong sign or index, or a transposed operand fails one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2603_08386_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
D9 = synth.HZ_DENOM


# --------------------------------------------------------------------------
# Table 2
# --------------------------------------------------------------------------

def test_table2_defaults_match_paper():
    g = json.load(open(os.path.join(GOLDEN, "table2.json")))
    for k, v in oracle.TABLE2.items():
        assert g[k]["final"] == v, k
        lo, hi = g[k]["range"]
        assert lo <= v <= hi


# --------------------------------------------------------------------------
# binning (Sec. 3.5): stable sort by pixel key, validity filter
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bin_matches_numpy_stable_sort(seed):
    s = synth.small_scene(seed, W=37, H=23, n_noise=6000, drone_px=60, extra_invalid=400)
    W, H = s.W, s.H
    b = oracle.bin_events(W, H, s.x, s.y, s.t, s.p, s.t0, s.window_us)
    x, y, t, p = (a.astype(np.int64) for a in (s.x, s.y, s.t, s.p))
    ok = (x >= 0) & (x < W) & (y >= 0) & (y < H) & (t >= s.t0) & (t < s.t0 + s.window_us) \
        & ((p == 1) | (p == -1))
    key = (y * W + x)[ok]
    order = np.argsort(key, kind="stable")
    assert b["n_valid"] == int(ok.sum())
    assert b["n_dropped"] == s.n - int(ok.sum())
    np.testing.assert_array_equal(b["tau"], (t[ok] - s.t0)[order])
    np.testing.assert_array_equal(b["pol"], p[ok][order])
    np.testing.assert_array_equal(b["counts"], np.bincount(key, minlength=W * H))
    np.testing.assert_array_equal(b["offsets"][1:], np.cumsum(np.bincount(key, minlength=W * H)))


def test_bin_polarity_01_and_edges():
    W, H, t0, win = 4, 3, 100, 50
    x = np.array([0, 3, 3, 4, 0, 1, 2, 0], np.int16)
    y = np.array([0, 2, 2, 0, -1, 1, 1, 0], np.int16)
    t = np.array([100, 149, 150, 120, 120, 99, 100, 101], np.int64)
    p = np.array([1, 0, 1, 1, 1, 1, 0, 2], np.int8)
    b = oracle.bin_events(W, H, x, y, t, p, t0, win, polarity_01=True)
    # kept: (0,0,t=100,+1), (3,2,t=149,-1), (2,1,t=100,-1); dropped: t=150, x=4, y=-1, t=99, p=2
    assert b["n_valid"] == 3 and b["n_dropped"] == 5
    assert b["counts"][0] == 1 and b["counts"][2 * W + 3] == 1 and b["counts"][1 * W + 2] == 1
    np.testing.assert_array_equal(b["tau"], [0, 0, 49])
    np.testing.assert_array_equal(b["pol"], [1, -1, -1])


def test_bin_empty():
    b = oracle.bin_events(5, 5, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), 0, 10)
    assert b["n_valid"] == 0 and b["n_dropped"] == 0
    assert np.all(b["offsets"] == 0)


# --------------------------------------------------------------------------
# NDFT power (Sec. 3.3 Eq. 6)
# --------------------------------------------------------------------------

def _rand_events(rng, n, window_us=20_000):
    tau = rng.integers(0, window_us, n).astype(np.int64)
    pol = rng.choice(np.array([-1, 1], np.int8), n)
    return tau, pol


def test_ndft_dc_is_square_of_polarity_sum():
    rng = np.random.default_rng(5)
    for n in (1, 7, 50, 333):
        tau, pol = _rand_events(rng, n)
        P = oracle.ndft(tau, pol, 0, 10_000, D9, 8)
        assert P[0] == float(int(pol.astype(np.int64).sum()) ** 2)


def test_ndft_uniform_times_is_the_dft():
    # tau_k = k * 1 ms, n = 1000 -> 1 Hz grid is exactly the n-point DFT
    rng = np.random.default_rng(6)
    n = 1000
    tau = np.arange(n, dtype=np.int64) * 1000
    pol = rng.choice(np.array([-1, 1], np.int8), n)
    P = oracle.ndft(tau, pol, 0, 1000, D9, n)
    ref = np.abs(np.fft.fft(pol.astype(np.float64))) ** 2
    np.testing.assert_allclose(P, ref, rtol=0, atol=1e-9 * ref.max())


def test_ndft_time_shift_invariance():
    rng = np.random.default_rng(7)
    tau, pol = _rand_events(rng, 40)
    P0 = oracle.ndft(tau, pol, 0, 2000, D9, 300)
    for c in (1, 12_345, 1 << 33, (1 << 40) - 7):
        P1 = oracle.ndft(tau + c, pol, 0, 2000, D9, 300)
        np.testing.assert_allclose(P1, P0, rtol=0, atol=1e-9 * P0.max())


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_ndft_pairwise_bruteforce(n):
    # |sum_k p_k e^{-i th_k}|^2 = sum_a sum_b p_a p_b cos(th_a - th_b), with the
    # phase difference taken exactly as a rational number of cycles.
    rng = np.random.default_rng(100 + n)
    tau, pol = _rand_events(rng, n)
    a0, da, nb = 3_000, 7_000, 40
    P = oracle.ndft(tau, pol, a0, da, D9, nb)
    for j in range(nb):
        a = a0 + j * da
        tot = 0.0
        for i in range(n):
            for k in range(n):
                cyc = Fraction(a * (int(tau[i]) - int(tau[k])), D9)
                frac = cyc - math.floor(cyc)
                tot += int(pol[i]) * int(pol[k]) * math.cos(2 * math.pi * float(frac))
        assert abs(P[j] - tot) <= 1e-9 * max(1.0, n * n)


def test_ndft_periodic_train_peaks_at_harmonics():
    # one +1 event per period T = 5 ms (200 Hz): P(m*200 Hz) = n^2, smaller elsewhere
    n, T = 20, 5000
    tau = np.arange(n, dtype=np.int64) * T + 137
    pol = np.ones(n, np.int8)
    P = oracle.ndft(tau, pol, 0, 10_000, D9, 200)  # 0..1990 Hz, 10 Hz step
    harm = np.arange(0, 200, 20)
    np.testing.assert_allclose(P[harm], n * n, rtol=1e-12)
    other = np.setdiff1d(np.arange(200), harm)
    assert P[other].max() < 0.5 * n * n


@pytest.mark.parametrize("duty", [0.2, 0.25, 0.37])
def test_ndft_rect_wave_harmonic_envelope(duty):
    # event-domain Eq. 1-5: +1 at kT, -1 at kT + duty*T gives
    # P(m f0) = |n (1 - e^{-2 pi i m duty})|^2 = 4 n^2 sin^2(pi m duty)
    n, T = 30, 10_000  # f0 = 100 Hz
    start = np.arange(n, dtype=np.int64) * T
    off = int(round(duty * T))
    tau = np.concatenate([start, start + off])
    pol = np.concatenate([np.ones(n, np.int8), -np.ones(n, np.int8)])
    P = oracle.ndft(tau, pol, 0, 100_000, D9, 12)  # bins at m * 100 Hz
    m = np.arange(12)
    ref = 4 * n * n * np.sin(np.pi * m * off / T) ** 2
    np.testing.assert_allclose(P, ref, rtol=0, atol=1e-9 * n * n)


def test_ndft_mode_grid_is_papers_normalised_form():
    # Sec. 3.5: timestamps normalised to [-pi, pi), integer modes k, F_k = sum p e^{i k t}
    rng = np.random.default_rng(9)
    win = 20_000
    tau, pol = _rand_events(rng, 64, win)
    K = 60
    P = oracle.ndft(tau, pol, 0, 1, win, K)
    tn = -np.pi + 2 * np.pi * tau.astype(np.float64) / win
    ref = np.abs(np.exp(1j * np.outer(np.arange(K), tn)) @ pol.astype(np.float64)) ** 2
    np.testing.assert_allclose(P, ref, rtol=0, atol=1e-9 * ref.max())
    # and it is the Hz grid with step 1/window = 50 Hz
    P2 = oracle.ndft(tau, pol, 0, 50_000, D9, K)
    np.testing.assert_allclose(P2, P, rtol=0, atol=1e-9 * ref.max())


def test_ndft_returns_complex_spectrum():
    rng = np.random.default_rng(10)
    tau, pol = _rand_events(rng, 25)
    P, F = oracle.ndft(tau, pol, 0, 3000, D9, 50, return_f=True)
    f = np.arange(50) * 3.0
    ref = np.exp(-2j * np.pi * np.outer(f, tau * 1e-6)) @ pol.astype(np.float64)
    np.testing.assert_allclose(F, ref, atol=1e-8)
    np.testing.assert_allclose(P, np.abs(F) ** 2, rtol=1e-12)


def test_ndft_at_matches_grid_and_derivative():
    rng = np.random.default_rng(11)
    tau, pol = _rand_events(rng, 30)
    Pg, Fg = oracle.ndft(tau, pol, 0, 2000, D9, 40, return_f=True)
    F, D = oracle.ndft_at(tau, pol, np.arange(40) * 2.0)
    np.testing.assert_allclose(F, Fg, atol=1e-9)
    # D = dF/df by central differences
    f = np.array([12.3456, 150.0, 333.0007])
    h = 1e-4
    Fp, _ = oracle.ndft_at(tau, pol, f + h, tau_c=10_000.0)
    Fm, _ = oracle.ndft_at(tau, pol, f - h, tau_c=10_000.0)
    _, D = oracle.ndft_at(tau, pol, f, tau_c=10_000.0)
    np.testing.assert_allclose(D, (Fp - Fm) / (2 * h), rtol=1e-6, atol=1e-6)


# --------------------------------------------------------------------------
# spectral flatness (Eq. 7)
# --------------------------------------------------------------------------

def test_sf_constant_spectrum_is_one():
    assert abs(oracle.log_sf(np.full(100, 3.7))) < 1e-14


def test_sf_two_level_closed_form():
    a, b = 2.0, 8.0
    P = np.array([a, b] * 50)
    ref = math.log(math.sqrt(a * b) / ((a + b) / 2))
    assert abs(oracle.log_sf(P) - ref) < 1e-14


def test_sf_of_random_phase_spectrum_is_exp_minus_gamma():
    # many random events -> P_j ~ exponential -> SF -> exp(-gamma) (statistical)
    rng = np.random.default_rng(12)
    vals = []
    for _ in range(8):
        tau, pol = _rand_events(rng, 400, 200_000)
        P = oracle.ndft(tau, pol, 1000, 5000, D9, 600)
        vals.append(oracle.log_sf(P))
    assert abs(np.mean(vals) - (-0.5772156649)) < 0.05


def test_sf_zero_power_reading():
    assert oracle.log_sf(np.zeros(10)) == 0.0


# --------------------------------------------------------------------------
# comb score (Eq. 8-11), hand-built spectra
# --------------------------------------------------------------------------

def test_comb_single_comb():
    P = np.ones(100)
    P[[10, 20, 30, 40]] = 5.0
    s, w = oracle.comb(P, M=4, d=0, h_min=4)
    assert (s, w) == (5.0, 10)


def test_comb_median_ignores_second_rotor():
    # a second fundamental at 13 raises the mean of the complement but not its median
    P = np.ones(100)
    P[[10, 20, 30, 40]] = 5.0
    P[[13, 26, 39, 52]] = 3.0
    s, w = oracle.comb(P, M=4, d=0, h_min=4)
    assert (s, w) == (5.0, 10)


def test_comb_window_max_and_union():
    # peaks offset inside the +-d window are found; H is the union of windows
    P = np.ones(120)
    P[[11, 19, 31, 42]] = [4.0, 6.0, 8.0, 10.0]
    s, w = oracle.comb(P, M=4, d=2, h_min=4)
    assert w == 10 and s == pytest.approx((4 + 6 + 8 + 10) / 4.0)


def test_comb_band_edge_m_valid():
    P = np.ones(50)
    P[[12, 24, 36, 48]] = 9.0
    # 4*12 + 2 > 49: only 3 harmonics in band -> invalid with h_min = 4
    s, w = oracle.comb(P, M=4, d=2, h_min=4)
    assert w != 12
    s, w = oracle.comb(P, M=4, d=2, h_min=3)
    assert w == 12 and s == pytest.approx(9.0)


def test_comb_even_median_and_zero_background():
    # N = 24, harmonics of w = 5 at {5, 10, 15, 20}; the 20 other bins hold ten 1s
    # and ten 3s, so the complement median is (1 + 3) / 2 = 2 and SNR = 10 / 2 = 5.
    P = np.array([1.0, 3.0] * 12)
    P[[5, 10, 15, 20]] = 10.0
    rest = np.delete(P, [5, 10, 15, 20])
    assert (rest == 1.0).sum() == 10 and (rest == 3.0).sum() == 10
    s, w = oracle.comb(P, M=4, d=0, h_min=4)
    assert (s, w) == (5.0, 5)
    s32, w32 = oracle.comb_f32(P.astype(np.float32), M=4, d=0, h_min=4)
    assert (float(s32), w32) == (5.0, 5)
    # zero background -> +inf
    Z = np.zeros(40)
    Z[[5, 10, 15, 20]] = 1.0
    s, w = oracle.comb(Z, M=4, d=0, h_min=4)
    assert math.isinf(s) and w == 5


def test_comb_tie_takes_first_candidate():
    P = np.ones(100)
    P[[10, 20, 30, 40, 50, 60, 70, 80]] = 5.0
    s, w = oracle.comb(P, M=4, d=0, h_min=4)
    assert w == 10  # w = 10 and w = 20 (20,40,60,80) both score 5, first wins


def test_comb_f32_equals_f64_on_exact_values():
    rng = np.random.default_rng(13)
    for _ in range(20):
        P = rng.integers(1, 64, 150).astype(np.float64)
        P[[7, 14, 21, 28]] = 200.0
        s64, w64 = oracle.comb(P, M=4, d=1, h_min=4)
        s32, w32 = oracle.comb_f32(P.astype(np.float32), M=4, d=1, h_min=4)
        assert w32 == w64
        assert abs(float(s32) - s64) <= 1e-6 * s64


def test_comb_bruteforce_small():
    # exhaustive restatement of Eq. 8-11 by numpy on random small spectra
    rng = np.random.default_rng(14)
    for trial in range(30):
        N = int(rng.integers(12, 60))
        M, d, hmin = int(rng.integers(1, 5)), int(rng.integers(0, 3)), 1
        P = rng.exponential(1.0, N)
        best, bw = -1.0, -1
        for w in range(max(1, d), N):
            ms = [m for m in range(1, M + 1) if m * w + d <= N - 1]
            if not ms:
                continue
            Hset = sorted({k for m in ms for k in range(m * w - d, m * w + d + 1)})
            if len(Hset) >= N:
                continue
            nw = np.mean([P[m * w - d:m * w + d + 1].max() for m in ms])
            B = np.median(np.delete(P, Hset))
            snr = nw / B
            if bw < 0 or snr > best:
                best, bw = snr, w
        s, w = oracle.comb(P, M=M, d=d, h_min=hmin)
        assert w == bw
        if bw >= 0:
            assert s == pytest.approx(best, rel=1e-12)


# --------------------------------------------------------------------------
# CCL and boxes (Sec. 3.5, Eq. 12)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_ccl8_matches_scipy(seed):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(seed)
    W, H = 61, 47
    mask = (rng.random((H, W)) < [0.2, 0.45, 0.6, 0.05][seed - 1]).astype(np.uint8)
    lab, n = oracle.ccl8(mask, W, H)
    ref, nref = ndimage.label(mask, structure=np.ones((3, 3)))
    assert n == nref
    lab = lab.reshape(H, W)
    for c in range(1, nref + 1):
        idx = np.flatnonzero(ref.ravel() == c)
        assert np.all(lab.ravel()[idx] == idx.min())
    assert np.all(lab[mask == 0] == -1)


def test_ccl8_diagonal_chain_is_one_component():
    W = H = 6
    mask = np.eye(6, dtype=np.uint8)[::-1].copy()  # anti-diagonal: 8- but not 4-connected
    lab, n = oracle.ccl8(mask, W, H)
    assert n == 1 and set(lab[lab >= 0]) == {5}


def _label_boxes(W, H, rects):
    m = np.zeros((H, W), np.uint8)
    for x0, y0, x1, y1 in rects:
        m[y0:y1 + 1, x0:x1 + 1] = 1
    lab, _ = oracle.ccl8(m, W, H)
    return lab


def test_boxes_area_filter_boundary():
    W, H = 100, 100
    lab = _label_boxes(W, H, [(0, 0, 13, 9), (50, 50, 72, 55), (30, 80, 30 + 145, 80)][:2]
                       + [(30, 80, 30 + 72, 81)])
    # areas: 14*10 = 140 (<147, dropped), 23*6 = 138 (dropped), 73*2 = 146 (dropped)
    assert oracle.boxes(lab, W, H, A_min=147, alpha=0.1).shape[0] == 0
    lab = _label_boxes(W, H, [(0, 0, 48, 2)])  # 49*3 = 147 kept
    bx = oracle.boxes(lab, W, H, A_min=147, alpha=0.1)
    assert bx.tolist() == [[0, 0, 48, 2, 147]]


def test_boxes_eq12_threshold_both_sides():
    # two 3x3 boxes (max dim 3); centroid distance 30 -> merge iff alpha*3 > 30
    W, H = 80, 10
    lab = _label_boxes(W, H, [(0, 0, 2, 2), (30, 0, 32, 2)])
    kept = oracle.boxes(lab, W, H, A_min=1, alpha=10.0)  # 30 < 30 is false
    assert kept.shape[0] == 2
    merged = oracle.boxes(lab, W, H, A_min=1, alpha=10.0 + 1e-9)
    assert merged.tolist() == [[0, 0, 32, 2, 18]]


def test_boxes_transitive_and_fixed_point():
    # A-B close, B-C close, A-C far: one group. Then the union box is close to D.
    W, H = 200, 20
    rects = [(0, 0, 1, 1), (10, 0, 11, 1), (20, 0, 21, 1), (40, 0, 41, 1)]
    lab = _label_boxes(W, H, rects)
    # pairwise: dist 10 between neighbours, alpha*2 = 12 -> A-B, B-C merge; C-D: 20 > 12
    # second merge pass: union box (0..21, 0..1) has max dim 22 -> alpha*22 = 132 > dist to D
    bx = oracle.boxes(lab, W, H, A_min=1, alpha=6.0)
    assert bx.tolist() == [[0, 0, 41, 1, 16]]


def test_boxes_sorted_output():
    W, H = 60, 60
    lab = _label_boxes(W, H, [(40, 5, 44, 9), (1, 30, 5, 34), (1, 5, 5, 9)])
    bx = oracle.boxes(lab, W, H, A_min=1, alpha=0.5)
    assert bx[:, :4].tolist() == [[1, 5, 5, 9], [40, 5, 44, 9], [1, 30, 5, 34]]


# --------------------------------------------------------------------------
# soft comb and its gradients (differentiation pattern)
# --------------------------------------------------------------------------

def test_softcomb_gradients_match_finite_differences():
    rng = np.random.default_rng(15)
    tau, pol = _rand_events(rng, 40, 40_000)
    kw = dict(delta=2.0, Q=3, B=7.5, tau_c=20_000.0)
    w = rng.uniform(0.5, 1.5, 6)
    sg = rng.uniform(1.0, 3.0, 6)
    f0 = 121.37
    r = oracle.softcomb(tau, pol, f0, w, sg, **kw)
    h = 1e-3
    sp = oracle.softcomb(tau, pol, f0 + h, w, sg, **kw)["S"]
    sm = oracle.softcomb(tau, pol, f0 - h, w, sg, **kw)["S"]
    assert r["dS_df0"] == pytest.approx((sp - sm) / (2 * h), rel=1e-6, abs=1e-9)
    for i in range(6):
        e = np.zeros(6)
        e[i] = 1e-5
        gw = (oracle.softcomb(tau, pol, f0, w + e, sg, **kw)["S"]
              - oracle.softcomb(tau, pol, f0, w - e, sg, **kw)["S"]) / 2e-5
        gs = (oracle.softcomb(tau, pol, f0, w, sg + e, **kw)["S"]
              - oracle.softcomb(tau, pol, f0, w, sg - e, **kw)["S"]) / 2e-5
        assert r["dS_dw"][i] == pytest.approx(gw, rel=1e-7, abs=1e-10)
        assert r["dS_dsigma"][i] == pytest.approx(gs, rel=1e-6, abs=1e-9)
    # the per-frequency gradients sum (with the chain factor h) to dS/df0
    tot = sum((hh + 1) * r["dS_df"][hh].sum() for hh in range(6))
    assert tot == pytest.approx(r["dS_df0"], rel=1e-10)


def test_softcomb_is_weighted_power_over_background():
    rng = np.random.default_rng(16)
    tau, pol = _rand_events(rng, 20, 40_000)
    # sigma -> tiny: only q = 0 carries weight, S = sum_h w_h P(h f0) / B
    w = np.arange(1, 7, dtype=np.float64)
    r = oracle.softcomb(tau, pol, 50.0, w, np.full(6, 1e-3), delta=2.0, Q=2, B=3.0)
    P = oracle.ndft(tau, pol, 50_000, 50_000, D9, 7)  # bins h*50 Hz, h = 1..7
    assert r["S"] == pytest.approx(float(np.dot(w, P[:6])) / 3.0, rel=1e-12)


# --------------------------------------------------------------------------
# whole window on C1 (sanity of the composition; not a pin on its own)
# --------------------------------------------------------------------------

def test_classify_composition_on_small_scene():
    s = synth.small_scene(21, W=40, H=32, n_noise=4000, drone_px=80, f0_hz=150.0,
                          grid=synth.hz_grid(0, 10, 100))
    b = oracle.bin_events(s.W, s.H, s.x, s.y, s.t, s.p, s.t0, s.window_us)
    c = oracle.classify(s.W, s.H, b, s.grid)
    # each classified pixel agrees with the per-function oracle
    for i in range(0, len(c["active"]), 37):
        k = c["active"][i]
        o0, o1 = b["offsets"][k], b["offsets"][k + 1]
        P = oracle.ndft(b["tau"][o0:o1], b["pol"][o0:o1], *s.grid)
        assert c["log_sf"][i] == pytest.approx(oracle.log_sf(P), abs=1e-12)
        if c["log_sf"][i] <= math.log(0.89):
            sn, w = oracle.comb(P)
            assert (c["snr"][i], c["w"][i]) == (pytest.approx(sn), w)
    assert np.all(b["counts"][c["active"]] >= 6)
    assert int((b["counts"] >= 6).sum()) == len(c["active"])


def test_ndft_at_negative_frequency_is_conjugate():
    # real polarities: F(-f) = conj(F(f)); pins the residue of a negative mHz count
    rng = np.random.default_rng(17)
    tau, pol = _rand_events(rng, 25)
    f = np.array([0.5, 13.25, 151.0007])
    Fp, Dp = oracle.ndft_at(tau, pol, f)
    Fm, Dm = oracle.ndft_at(tau, pol, -f)
    np.testing.assert_allclose(Fm, np.conj(Fp), atol=1e-9)
    np.testing.assert_allclose(Dm, -np.conj(Dp), atol=1e-6)  # D(-f) = -conj(D(f))


def test_box_frequencies_hand_case():
    # 5x4 sensor; rotor pixels (x, y): (1,1) snr 3 bin 7, (3,1) snr 5 bin 9,
    # (2,2) snr 5 bin 4 (ties with (3,1): key 8 < 12 wins in a box holding both),
    # (4,3) snr 9 bin 2 but masked off; a box with no rotor pixel gives -1
    W = 5
    active = np.array([6, 8, 12, 19], np.int64)          # (1,1), (3,1), (2,2), (4,3)
    mask = np.zeros(20, np.uint8)
    mask[[6, 8, 12]] = 1
    snr = np.array([3.0, 5.0, 5.0, 9.0], np.float32)
    f0 = np.array([7, 9, 4, 2], np.int32)
    boxes = np.array([[0, 0, 4, 3, 0],    # everything: tie 5.0 at keys 8 and 12 -> key 8
                      [0, 0, 1, 1, 0],    # only (1,1)
                      [2, 2, 4, 3, 0],    # (2,2) rotor, (4,3) not
                      [0, 3, 3, 3, 0]])   # no rotor pixel
    fb, sb = oracle.box_frequencies(boxes, active, mask, snr, f0, W)
    np.testing.assert_array_equal(fb, [9, 7, 4, -1])
    np.testing.assert_array_equal(sb, np.float32([5.0, 3.0, 5.0, 0.0]))
    # lower medians of the rotor bins (7, 9, 4 -> sorted 4, 7, 9 -> 7; 7; 4; none)
    # on a 2 Hz grid from 0 (bin j = 2 j Hz)
    med = oracle.box_median_hz(boxes, active, mask, f0, W, (0, 2000, 1_000_000_000, 750))
    np.testing.assert_array_equal(med, np.float32([14.0, 14.0, 8.0, 0.0]))
    two = oracle.box_median_hz(np.array([[1, 1, 3, 1, 0]]), active, mask, f0, W,
                               (0, 2000, 1_000_000_000, 750))
    np.testing.assert_array_equal(two, np.float32([14.0]))  # bins 7, 9: lower median 7


def test_ndft_f32_agrees_with_fp64():
    # the FP32 CPU baseline computes Eq. 6 to FP32 accuracy: P(0) = (sum p)^2
    # exactly for small n, and within 1e-5 of each row's peak of the FP64 sum
    rng = np.random.default_rng(17)
    for n in (1, 7, 40, 300):
        tau = np.sort(rng.integers(0, 30_000, n)).astype(np.int64)
        pol = rng.choice(np.array([-1, 1], np.int8), n)
        P64 = oracle.ndft(tau, pol, 0, 2000, 1_000_000_000, 750)
        P32 = oracle.ndft_f32(tau, pol, 0, 2000, 1_000_000_000, 750)
        assert P32[0] == np.float32(float(pol.sum()) ** 2)
        assert np.abs(P32 - P64).max() <= 1e-5 * P64.max()
