"""The hybrid route's approximation (DDHF_FORM_HYBRID, footnote to Sec. 3.3)
checked on the CPU against the oracle's exact Eq. 6, with the parameters the
library uses: centre-bin phase shift, grid spacing s = floor(D / (2 da N)),
an 8-point exponential-of-semicircle kernel with beta = 2.30 * 8 (Barnett,
Magland and af Klinteberg 2019) and deconvolution by its Fourier transform,
here evaluated by scipy's adaptive quadrature (independent of the library's
Simpson rule). The bound this pins, 1e-6 of the pixel's peak power, is two
orders of magnitude inside the 1e-4 parity bar the GPU tests apply."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2603_08386_gb300 import synth

W_PTS, BETA = 8, 2.30 * 8


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def es(z):
    x = np.clip(1.0 - (2.0 * z / W_PTS) ** 2, 0.0, None)
    return np.exp(BETA * (np.sqrt(x) - 1.0))


def es_hat(kappa):
    f = lambda z: float(es(np.array(z))) * math.cos(2 * math.pi * kappa * z)
    v, _ = integrate.quad(f, -W_PTS / 2, W_PTS / 2, limit=200, epsabs=1e-13, epsrel=1e-12)
    return v


def hybrid_power(tau, pol, grid, window_us):
    a0, da, D, N = grid
    s = D // (2 * da * N)
    J = N // 2
    ac = a0 + J * da
    tau = np.asarray(tau, np.int64)
    q = pol * np.exp(-2j * np.pi * ((ac * tau) % D) / D)
    i0 = tau // s
    fr = (tau - i0 * s) / s
    G = (window_us - 1) // s + W_PTS
    c = np.zeros(G, complex)
    for i in range(W_PTS):
        np.add.at(c, i0 + i, q * es((i - (W_PTS // 2 - 1)) - fr))
    m = np.arange(N, dtype=np.int64) - J
    tg = (np.arange(G, dtype=np.int64) - (W_PTS // 2 - 1)) * s
    r = (np.outer(tg, m) % D) * da % D
    dec = np.array([1.0 / es_hat(k * da * s / D) for k in m])
    F = c @ (np.exp(-2j * np.pi * r / D) * dec[None, :])
    return np.abs(F) ** 2, s, G


@pytest.mark.parametrize("grid,window_us,n,seed", [
    (synth.hz_grid(0, 2, 750), 30_000, 3000, 1),      # C3's grid
    (synth.hz_grid(0, 2, 750), 30_000, 40, 2),        # few events
    (synth.hz_grid(97.5, 1.5, 600), 30_000, 800, 3),  # band away from 0 Hz
    (synth.hz_grid(0, 1, 2000), 50_000, 1500, 4),     # C2's grid
    (synth.mode_grid(20_000, 100), 20_000, 500, 5),   # the paper's modes
])
def test_spread_and_deconvolve_within_1e6_of_eq6(grid, window_us, n, seed):
    rng = np.random.default_rng(seed)
    tau = np.sort(rng.integers(0, window_us, n))
    pol = rng.choice([-1.0, 1.0], n)
    P, s, G = hybrid_power(tau, pol, grid, window_us)
    ref = oracle.ndft(tau.astype(np.int64), pol.astype(np.int8), *grid)
    err = np.abs(P - ref).max() / ref.max()
    assert s >= 1 and G <= 1024
    assert err <= 1e-6, err


def test_periodic_train_peak_through_the_grid():
    # a 100 Hz train of n events, one per 10 ms period: P(100 m Hz) = n^2 for
    # every harmonic (Eq. 6 closed form), also through the spread/deconvolve route
    grid = synth.hz_grid(0, 2, 750)
    n = 3
    tau = np.arange(n, dtype=np.int64) * 10_000 + 17
    P, _, _ = hybrid_power(tau, np.ones(n), grid, 30_000)
    for m in range(0, 8):
        assert P[50 * m] == pytest.approx(n * n, rel=1e-6)
    ref = oracle.ndft(tau, np.ones(n, np.int8), *grid)
    assert np.abs(P - ref).max() <= 1e-6 * ref.max()


def test_kernel_transform_quadratures_agree():
    # the library integrates in theta (z = (w/2) sin theta) by Simpson's rule;
    # the same rule here against scipy's adaptive quadrature in z
    th = np.linspace(-np.pi / 2, np.pi / 2, 2049)
    wts = np.ones(2049)
    wts[1:-1:2], wts[2:-1:2] = 4, 2
    for kappa in (0.0, 0.1, 0.25, 0.75, 1.25):
        f = np.exp(BETA * (np.cos(th) - 1)) * np.cos(th) * (W_PTS / 2) * \
            np.cos(2 * np.pi * kappa * (W_PTS / 2) * np.sin(th))
        simpson = (wts * f).sum() * (th[1] - th[0]) / 3
        assert simpson == pytest.approx(es_hat(kappa), rel=1e-10, abs=1e-14)


@pytest.mark.parametrize("grid,window_us,hybrid_min", [
    (synth.hz_grid(0, 2, 750), 30_000, 128),
    (synth.hz_grid(0, 1, 2000), 50_000, 32),
    (synth.hz_grid(0, 10, 100), 20_000, 16),
    (synth.hz_grid(97.5, 1.5, 600), 30_000, 300),
    (synth.mode_grid(20_000, 100), 20_000, 64),
])
def test_library_geometry_and_deconvolution(grid, window_us, hybrid_min):
    # the library's own plan (host code, no device) follows the stated rule,
    # and its deconvolution factors equal 1 / psi^ by scipy's quadrature
    from paper_2603_08386_gb300 import ddhf
    st, s, G, thr, dec = ddhf.ddhf_hybrid_geometry(grid, window_us, hybrid_min)
    a0, da, D, N = grid
    assert s == D // (2 * da * N)
    assert G == (window_us - 1) // s + W_PTS
    assert st == 0 and thr == max(hybrid_min, 16, -(-G // 2))
    J = N // 2
    for j in sorted({0, 1, J - 1, J, J + 1, N - 2, N - 1, N // 3}):
        want = 1.0 / es_hat((j - J) * da * s / D)
        assert dec[j] == pytest.approx(want, rel=2e-7)
    np.testing.assert_array_equal(dec[J - 1::-1][: N - 1 - J], dec[J + 1:][: J])  # even in m


def test_library_geometry_refuses_windows_off_the_route():
    from paper_2603_08386_gb300 import ddhf
    g = synth.hz_grid(0, 2, 750)
    st, s, G, thr, _ = ddhf.ddhf_hybrid_geometry(g, 400_000, 64)  # G = 1209 > 1024
    assert (st, s, G, thr) == (5, 333, 1209, 0)
    st, _, G, thr, _ = ddhf.ddhf_hybrid_geometry(g, 2_000, 64)    # G = 14 < 16
    assert (st, G, thr) == (5, 14, 0)
    st, s, _, thr, _ = ddhf.ddhf_hybrid_geometry(synth.mode_grid(20_000, 16384), 20_000, 64)
    assert (st, s, thr) == (5, 0, 0)                               # spacing below 1 us
    assert ddhf.ddhf_hybrid_geometry(g, 30_000, 0)[0] == 1
    assert ddhf.ddhf_hybrid_geometry((0, 0, 10**9, 750), 30_000, 64)[0] == 1
