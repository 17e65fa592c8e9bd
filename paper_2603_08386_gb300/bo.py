"""Bayesian optimisation with a Gaussian-process surrogate and expected
improvement, as Sec. 4.1 uses it to tune the thresholds of Sec. 3.4-3.5:
uniform priors over box ranges (Table 2), a number of uniformly random
evaluation points first, then one point per iteration at the maximum of the
expected improvement.

Surrogate: zero-mean GP on the standardised objective over the unit cube,
Matern 5/2 kernel with one length scale per dimension (ARD), a signal
variance and a noise variance, fitted by maximising the log marginal
likelihood (L-BFGS-B on the log hyperparameters, analytic gradient).
Integer dimensions are rounded before evaluation and the rounded point is
what the surrogate sees. Host code (numpy, scipy); maximisation.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import linalg, optimize
from scipy.stats import norm

SQRT5 = math.sqrt(5.0)


def matern52(X1, X2, ls, s2):
    """s2 (1 + sqrt5 r + 5 r^2 / 3) exp(-sqrt5 r), r = |(x1 - x2) / ls|."""
    D = (X1[:, None, :] - X2[None, :, :]) / ls
    r = np.sqrt(np.maximum((D * D).sum(-1), 0.0))
    return s2 * (1.0 + SQRT5 * r + (5.0 / 3.0) * r * r) * np.exp(-SQRT5 * r)


class GP:
    """GP regression with a Matern 5/2 ARD kernel."""

    def __init__(self, dim):
        self.dim = dim
        self.theta = np.concatenate([np.log(np.full(dim, 0.3)), [0.0, math.log(1e-3)]])

    def _unpack(self, theta):
        return np.exp(theta[: self.dim]), math.exp(theta[self.dim]), math.exp(theta[self.dim + 1])

    def nll(self, theta, X, y):
        """Negative log marginal likelihood and its gradient in theta."""
        ls, s2, sn2 = self._unpack(theta)
        n = X.shape[0]
        D = (X[:, None, :] - X[None, :, :]) / ls
        D2 = D * D
        r = np.sqrt(np.maximum(D2.sum(-1), 0.0))
        e = np.exp(-SQRT5 * r)
        Kf = s2 * (1.0 + SQRT5 * r + (5.0 / 3.0) * r * r) * e
        K = Kf + (sn2 + 1e-10) * np.eye(n)
        try:
            L = linalg.cholesky(K, lower=True)
        except linalg.LinAlgError:
            return 1e25, np.zeros_like(theta)
        a = linalg.cho_solve((L, True), y)
        val = 0.5 * y @ a + np.log(np.diag(L)).sum() + 0.5 * n * math.log(2 * math.pi)
        W = np.outer(a, a) - linalg.cho_solve((L, True), np.eye(n))
        g = np.empty_like(theta)
        # dK/dlog ls_i = s2 (5/3) (1 + sqrt5 r) exp(-sqrt5 r) (d_i / ls_i)^2
        base = s2 * (5.0 / 3.0) * (1.0 + SQRT5 * r) * e
        for i in range(self.dim):
            g[i] = -0.5 * np.sum(W * (base * D2[:, :, i]))
        g[self.dim] = -0.5 * np.sum(W * Kf)
        g[self.dim + 1] = -0.5 * sn2 * np.trace(W)
        return float(val), g

    def fit(self, X, y, restarts=2, rng=None):
        self.X = np.asarray(X, np.float64)
        self.mu_y = float(np.mean(y))
        sd = float(np.std(y))
        self.sd_y = sd if sd > 0 else 1.0
        self.y = (np.asarray(y, np.float64) - self.mu_y) / self.sd_y
        bounds = [(math.log(1e-2), math.log(10.0))] * self.dim + \
                 [(math.log(1e-2), math.log(10.0)), (math.log(1e-6), math.log(1.0))]
        starts = [self.theta, np.concatenate([np.zeros(self.dim) + math.log(0.5), [0.0, -4.0]])]
        rng = rng or np.random.default_rng(0)
        for _ in range(max(0, restarts - 2)):
            starts.append(np.array([rng.uniform(lo, hi) for lo, hi in bounds]))
        best = None
        for t0 in starts:
            res = optimize.minimize(self.nll, np.clip(t0, [b[0] for b in bounds],
                                                      [b[1] for b in bounds]),
                                    args=(self.X, self.y), jac=True, method="L-BFGS-B",
                                    bounds=bounds, options=dict(maxiter=200))
            if best is None or res.fun < best.fun:
                best = res
        self.theta = best.x
        ls, s2, sn2 = self._unpack(self.theta)
        K = matern52(self.X, self.X, ls, s2) + (sn2 + 1e-10) * np.eye(len(self.X))
        self.L = linalg.cholesky(K, lower=True)
        self.alpha = linalg.cho_solve((self.L, True), self.y)
        return self

    def predict(self, Xs):
        """Posterior mean and standard deviation of the (unstandardised) objective."""
        ls, s2, _ = self._unpack(self.theta)
        Ks = matern52(self.X, np.asarray(Xs, np.float64), ls, s2)
        mu = Ks.T @ self.alpha
        v = linalg.solve_triangular(self.L, Ks, lower=True)
        var = np.maximum(s2 - (v * v).sum(0), 1e-12)
        return mu * self.sd_y + self.mu_y, np.sqrt(var) * self.sd_y


def expected_improvement(mu, sd, best, xi=0.01):
    """EI of a maximisation: E[max(f - best - xi, 0)] under N(mu, sd^2)."""
    imp = mu - best - xi
    z = imp / sd
    return imp * norm.cdf(z) + sd * norm.pdf(z)


class Space:
    """Box of named dimensions (name, lo, hi, is_int) and the unit-cube map."""

    def __init__(self, dims):
        self.dims = list(dims)
        self.lo = np.array([d[1] for d in self.dims], np.float64)
        self.hi = np.array([d[2] for d in self.dims], np.float64)
        self.is_int = np.array([bool(d[3]) for d in self.dims])

    def decode(self, u):
        v = self.lo + np.clip(u, 0.0, 1.0) * (self.hi - self.lo)
        v = np.where(self.is_int, np.rint(v), v)
        return {d[0]: (int(x) if d[3] else float(x)) for d, x in zip(self.dims, v)}

    def encode(self, vals):
        v = np.array([vals[d[0]] for d in self.dims], np.float64)
        return (v - self.lo) / np.where(self.hi > self.lo, self.hi - self.lo, 1.0)


def maximise(objective, space: Space, n_init=50, n_iter=300, seed=0, n_cand=2048,
             refit_every=5, log=None):
    """Maximise objective(dict) over the space: n_init uniform random points,
    then n_iter expected-improvement steps. Returns (best dict, best value,
    history list of (dict, value))."""
    rng = np.random.default_rng(seed)
    dim = len(space.dims)
    X, y, hist = [], [], []

    def evaluate(u):
        vals = space.decode(u)
        f = float(objective(vals))
        X.append(space.encode(vals))
        y.append(f)
        hist.append((vals, f))
        if log:
            log(len(hist), vals, f)

    for _ in range(n_init):
        evaluate(rng.random(dim))
    gp = GP(dim)
    for it in range(n_iter):
        Xa, ya = np.array(X), np.array(y)
        if it % refit_every == 0 or not hasattr(gp, "L"):
            gp.fit(Xa, ya, rng=rng)
        else:
            gp.X, gp.y = Xa, (ya - gp.mu_y) / gp.sd_y
            ls, s2, sn2 = gp._unpack(gp.theta)
            K = matern52(Xa, Xa, ls, s2) + (sn2 + 1e-10) * np.eye(len(Xa))
            gp.L = linalg.cholesky(K, lower=True)
            gp.alpha = linalg.cho_solve((gp.L, True), gp.y)
        best_i = int(np.argmax(ya))
        cand = np.concatenate([
            rng.random((n_cand, dim)),
            np.clip(Xa[best_i] + 0.05 * rng.standard_normal((n_cand // 4, dim)), 0.0, 1.0)])
        mu, sd = gp.predict(cand)
        ei = expected_improvement(mu, sd, float(ya[best_i]))
        evaluate(cand[int(np.argmax(ei))])
    b = int(np.argmax(y))
    return hist[b][0], y[b], hist
