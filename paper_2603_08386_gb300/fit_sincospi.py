"""Regenerate the polynomial coefficients of the kernels' sin(pi x) and
cos(pi x) (sincospi_reduced in csrc/ddhf_internal.cuh).

After the quadrant reduction the argument y lies in [-1/4, 1/4]; with t = y^2
the kernels evaluate
    sin(pi y) = y P(t),        P of degree 4,
    cos(pi y) = 1 + t C(t),    C of degree 3,
by Horner steps in FP32. The coefficients are weighted least-squares fits in
FP64 over a dense grid of y in (0, 1/4], weighted so that the residual is the
relative error of sin(pi y) and of cos(pi y), then rounded to FP32.

    python -m paper_2603_08386_gb300.fit_sincospi      # prints them
"""
from __future__ import annotations

import numpy as np


def fit(n_points: int = 200001):
    """(P, C): FP32 coefficients, lowest degree first."""
    y = np.linspace(1e-6, 0.25, n_points)
    t = y * y
    s = np.sin(np.pi * y)
    c = np.cos(np.pi * y)
    # sin: P(t) ~ sin(pi y) / y; the relative error of y P(t) is that of P
    a_s = np.stack([t ** k for k in range(5)], 1)
    b_s = s / y
    w_s = 1.0 / np.abs(b_s)
    p, *_ = np.linalg.lstsq(a_s * w_s[:, None], b_s * w_s, rcond=None)
    # cos: C(t) ~ (cos(pi y) - 1) / t; relative error of 1 + t C(t) = t (C - C*) / cos
    a_c = np.stack([t ** k for k in range(4)], 1)
    b_c = (c - 1.0) / t
    w_c = t / np.abs(c)
    q, *_ = np.linalg.lstsq(a_c * w_c[:, None], b_c * w_c, rcond=None)
    return p.astype(np.float32), q.astype(np.float32)


def max_rel_error(P, C, n_points: int = 100001):
    """Largest relative error of the FP64-evaluated polynomials on [-1/4, 1/4]."""
    y = np.linspace(-0.25, 0.25, n_points)
    t = y * y
    ps = np.polynomial.polynomial.polyval(t, P.astype(np.float64)) * y
    pc = 1.0 + t * np.polynomial.polynomial.polyval(t, C.astype(np.float64))
    s, c = np.sin(np.pi * y), np.cos(np.pi * y)
    nz = np.abs(s) > 0
    return float(np.max(np.abs(ps[nz] - s[nz]) / np.abs(s[nz]))), float(np.max(np.abs(pc - c) / c))


if __name__ == "__main__":
    P, C = fit()
    print("sin(pi y) = y P(y^2), P (highest degree first):",
          ", ".join(f"{float(v):.9g}f" for v in P[::-1]))
    print("cos(pi y) = 1 + y^2 C(y^2), C (highest degree first):",
          ", ".join(f"{float(v):.9g}f" for v in C[::-1]))
    print("max relative error (FP64 evaluation): sin %.3g, cos %.3g" % max_rel_error(P, C))
