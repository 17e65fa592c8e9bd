"""The labelling kernel's reduced set of unions gives the full 8-connected
components.

Each mask pixel of the CUDA labelling unites only with: the pixel above when
it is set; otherwise the left neighbour (or, without it, the upper-left one)
and the upper-right one. This file replays that rule with a plain sequential
union-find (roots linked to the smaller index, so labels are the minimum
linear index of each component) and compares the labels with the oracle's
breadth-first labelling, on random masks of many densities and on structured
ones whose pixels connect through diagonals only.
"""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def reduced_rule_labels(mask, W, H):
    par = np.where(mask.ravel() != 0, np.arange(W * H), -1)

    def find(a):
        while par[a] != a:
            a = par[a]
        return a

    def unite(a, b):
        a, b = find(a), find(b)
        if a != b:
            par[max(a, b)] = min(a, b)

    m = mask.reshape(H, W) != 0
    for y in range(H):
        for x in range(W):
            if not m[y, x]:
                continue
            i = y * W + x
            if y > 0 and m[y - 1, x]:
                unite(i, i - W)
            else:
                if x > 0 and m[y, x - 1]:
                    unite(i, i - 1)
                elif y > 0 and x > 0 and m[y - 1, x - 1]:
                    unite(i, i - W - 1)
                if y > 0 and x < W - 1 and m[y - 1, x + 1]:
                    unite(i, i - W + 1)
    return np.array([find(i) if par[i] >= 0 else -1 for i in range(W * H)], dtype=np.int64)


def _check(mask, W, H):
    ref, _ = oracle.ccl8(mask.astype(np.uint8).ravel(), W, H)
    np.testing.assert_array_equal(reduced_rule_labels(mask, W, H), np.asarray(ref, np.int64))


@pytest.mark.parametrize("density", [0.1, 0.3, 0.45, 0.55, 0.7, 0.9])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_reduced_unions_random_masks(density, seed):
    W, H = 23, 17
    mask = np.random.default_rng(seed).random((H, W)) < density
    _check(mask, W, H)


def test_reduced_unions_structured_masks():
    W, H = 29, 19
    yy, xx = np.mgrid[0:H, 0:W]
    for mask in ((xx + yy) % 2 == 0, (xx + yy) % 3 == 0, (xx - yy) % 4 == 0, yy % 2 == 0,
                 xx % 2 == 0, (xx % 2 == 0) & (yy % 2 == 0), np.ones((H, W), bool),
                 np.abs(xx - yy) == 0, np.abs(xx + yy - (H - 1)) == 0,
                 (xx % 5 == 0) | (yy % 4 == 0)):
        _check(mask, W, H)
