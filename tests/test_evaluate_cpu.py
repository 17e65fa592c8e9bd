"""Detection-quality metric and the Bayesian-optimisation search (Sec. 4.1,
4.2) on CPU: IoU against pixel-set counting, the one-to-one matching and F1
on hand cases, the GP's likelihood gradient against finite differences, its
interpolation, the expected-improvement closed form, and the search finding
known maxima (continuous and integer dimensions)."""
import math

import numpy as np
import pytest

from paper_2603_08386_gb300 import bo, evaluate


def pixel_iou(a, b):
    A = {(x, y) for x in range(a[0], a[2] + 1) for y in range(a[1], a[3] + 1)}
    B = {(x, y) for x in range(b[0], b[2] + 1) for y in range(b[1], b[3] + 1)}
    return len(A & B) / len(A | B)


def test_iou_hand_cases_and_pixel_sets():
    assert evaluate.box_iou((0, 0, 9, 9), (0, 0, 9, 9)) == 1.0
    assert evaluate.box_iou((0, 0, 9, 9), (10, 0, 19, 9)) == 0.0
    assert evaluate.box_iou((0, 0, 9, 9), (9, 0, 18, 9)) == pytest.approx(10 / 190)
    assert evaluate.box_iou((0, 0, 9, 9), (5, 0, 14, 9)) == pytest.approx(50 / 150)
    assert evaluate.box_iou((0, 0, 9, 9), (2, 2, 5, 5)) == pytest.approx(16 / 100)
    assert evaluate.box_iou((3, 3, 3, 3), (3, 3, 3, 3)) == 1.0
    rng = np.random.default_rng(1)
    for _ in range(300):
        a = sorted(rng.integers(0, 12, 2)), sorted(rng.integers(0, 12, 2))
        b = sorted(rng.integers(0, 12, 2)), sorted(rng.integers(0, 12, 2))
        A = (a[0][0], a[1][0], a[0][1], a[1][1])
        B = (b[0][0], b[1][0], b[0][1], b[1][1])
        assert evaluate.box_iou(A, B) == pytest.approx(pixel_iou(A, B))


def test_match_and_f1():
    g = [(0, 0, 9, 9)]
    assert evaluate.match([(0, 0, 9, 9), (1, 0, 9, 9)], g) == (1, 1, 0)
    assert evaluate.match([], g) == (0, 0, 1)
    assert evaluate.match([(0, 0, 9, 9)], []) == (0, 1, 0)
    # below the threshold: (0,0,9,9) vs (5,0,14,9) is 1/3
    assert evaluate.match([(5, 0, 14, 9)], g) == (0, 1, 1)
    assert evaluate.match([(5, 0, 14, 9)], g, thr=0.3) == (1, 0, 0)
    # greedy by IoU: p0 takes g0 (IoU 0.9) although p0-g1, p1-g0 would match both
    g2 = [(0, 0, 9, 9), (1, 0, 10, 9)]
    p2 = [(0, 0, 9, 8), (0, 0, 8, 9)]
    tp, fp, fn = evaluate.match(p2, g2)
    assert tp + fp == 2 and tp + fn == 2
    assert evaluate.f1_score(3, 1, 2) == pytest.approx(6 / 9)
    assert evaluate.f1_score(0, 0, 0) == 1.0
    assert evaluate.f1_score(0, 4, 0) == 0.0


def test_gp_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    X = rng.random((12, 3))
    y = np.sin(3 * X[:, 0]) + X[:, 1] ** 2 - X[:, 2]
    gp = bo.GP(3)
    th = np.array([math.log(0.4), math.log(0.7), math.log(0.2), 0.3, math.log(1e-2)])
    f0, g = gp.nll(th, X, y)
    for i in range(th.size):
        e = np.zeros_like(th)
        e[i] = 1e-6
        num = (gp.nll(th + e, X, y)[0] - gp.nll(th - e, X, y)[0]) / 2e-6
        assert g[i] == pytest.approx(num, rel=1e-4, abs=1e-6)


def test_gp_interpolates_and_ei_closed_form():
    X = np.linspace(0, 1, 9)[:, None]
    y = np.sin(4 * X[:, 0])
    gp = bo.GP(1).fit(X, y)
    mu, sd = gp.predict(X)
    np.testing.assert_allclose(mu, y, atol=2e-2)
    assert (sd < 0.1).all()
    mu2, sd2 = gp.predict(np.array([[0.0625]]))
    assert abs(mu2[0] - math.sin(0.25)) < 0.05
    assert bo.expected_improvement(np.array([1.0]), np.array([1.0]), 1.0, xi=0.0)[0] == \
        pytest.approx(1 / math.sqrt(2 * math.pi))
    assert bo.expected_improvement(np.array([3.0]), np.array([1e-9]), 1.0, xi=0.0)[0] == \
        pytest.approx(2.0)


def test_bo_finds_known_maxima():
    sp = bo.Space([("a", 0.0, 1.0, False), ("b", -2.0, 2.0, False)])
    f = lambda v: -((v["a"] - 0.3) ** 2 + 0.25 * (v["b"] - 0.8) ** 2)
    best, val, hist = bo.maximise(f, sp, n_init=8, n_iter=22, seed=1)
    assert len(hist) == 30
    assert abs(best["a"] - 0.3) < 0.08 and abs(best["b"] - 0.8) < 0.3
    sp2 = bo.Space([("k", 0, 10, True), ("x", 0.0, 1.0, False)])
    g = lambda v: -(v["k"] - 3) ** 2 - (v["x"] - 0.5) ** 2
    best2, val2, _ = bo.maximise(g, sp2, n_init=6, n_iter=20, seed=2)
    assert best2["k"] == 3 and isinstance(best2["k"], int)
    assert abs(best2["x"] - 0.5) < 0.15
    # integer dimensions are evaluated at rounded values only
    seen = {v["k"] for v, _ in bo.maximise(lambda v: float(v["k"]), sp2, 4, 4, seed=3)[2]}
    assert all(isinstance(k, int) for k in seen)
