"""Seeded synthetic workloads for the iterative Vecchia-Laplace hot path.

This module only draws inputs: locations, the random Vecchia ordering, a latent
field, responses and test locations. It holds none of the method's arithmetic
(no Vecchia factor, no Laplace approximation, no solver) and is imported both by
the tests (which hand the same inputs to the CPU oracle and to the CUDA path) and
by ``bench.py``. Random numbers that the method itself draws (SLQ probes,
simulation vectors) are not made here: each side generates them from the
published Philox4x64-10 definition.

Workload shapes follow the paper's simulation setting (Section 4.1: uniform
locations in the unit square, Matern-1.5 covariance, sigma^2 = 1, range 0.05,
Bernoulli-logit responses, random ordering, m = 20) and the larger stand-ins for
the satellite-swath data of Section 5 (a regular grid with rectangular gaps).

Latent fields
-------------
* ``exact``: b = chol(Sigma + 1e-10 I) eps, the textbook dense draw (n <= ~5000).
* ``rff``:   random Fourier features (Rahimi & Recht, 2007): b(s) =
  sigma * sqrt(2/K) * sum_k cos(w_k . s + phi_k) with w_k drawn from the spectral
  density of the covariance (a bivariate Student-t with 2*nu degrees of freedom
  scaled by sqrt(2 nu)/rho). Used for large n in place of a Vecchia m = 40 draw so
  that this module stays free of the method's arithmetic.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

COV_EXPONENTIAL = 0
COV_MATERN15 = 1
LIK_BERNOULLI_LOGIT = 0
LIK_POISSON_LOG = 1
LIK_GAMMA_LOG = 2


@dataclasses.dataclass
class Problem:
    """One latent-GP problem: everything a caller hands to the library."""

    name: str
    locs: np.ndarray          # (n, 2) float64, user order
    order: np.ndarray         # (n,) int32, order[k] = user index of the k-th point in the Vecchia order
    y: np.ndarray             # (n,) float64 responses, user order
    F: np.ndarray             # (n,) float64 fixed-effect offset, user order
    cov: int                  # COV_EXPONENTIAL | COV_MATERN15
    sigma2: float
    rho: float
    m: int
    lik: int                  # LIK_BERNOULLI_LOGIT | LIK_POISSON_LOG | LIK_GAMMA_LOG
    t: int = 50               # SLQ probes
    s: int = 100              # simulation vectors for predictive variances
    test_locs: np.ndarray | None = None   # (n_p, 2)
    Fp: np.ndarray | None = None          # (n_p,)
    b_true: np.ndarray | None = None      # latent draw (user order), for reference only
    seed: int = 1
    xi: float = 1.0                       # gamma shape (auxiliary likelihood parameter)
    X: np.ndarray | None = None           # (n, p) predictors of F = X beta, user order
    beta: np.ndarray | None = None        # (p,) coefficients that made F

    @property
    def n(self) -> int:
        return int(self.locs.shape[0])

    @property
    def nugget(self) -> float:
        return 1e-10 * self.sigma2


def _cov_textbook(h: np.ndarray, cov: int, sigma2: float, rho: float) -> np.ndarray:
    # Only used to draw the exact latent field for small n.
    if cov == COV_EXPONENTIAL:
        return sigma2 * np.exp(-h / rho)
    a = math.sqrt(3.0) * h / rho
    return sigma2 * (1.0 + a) * np.exp(-a)


def latent_exact(locs: np.ndarray, cov: int, sigma2: float, rho: float, rng) -> np.ndarray:
    d = locs[:, None, :] - locs[None, :, :]
    K = _cov_textbook(np.sqrt((d * d).sum(-1)), cov, sigma2, rho)
    K[np.diag_indices_from(K)] += 1e-10 * sigma2
    return np.linalg.cholesky(K) @ rng.standard_normal(len(locs))


def latent_rff(locs: np.ndarray, cov: int, sigma2: float, rho: float, rng, K: int = 0) -> np.ndarray:
    K = K or (512 if len(locs) <= 200_000 else 256)
    nu = 0.5 if cov == COV_EXPONENTIAL else 1.5
    g = rng.standard_normal((K, 2))
    u = rng.chisquare(2.0 * nu, size=K)
    w = (math.sqrt(2.0 * nu) / rho) * g / np.sqrt(u / (2.0 * nu))[:, None]
    phi = rng.uniform(0.0, 2.0 * math.pi, size=K)
    b = np.empty(len(locs))
    step = 65536
    for a in range(0, len(locs), step):
        arg = locs[a:a + step] @ w.T + phi
        b[a:a + step] = np.cos(arg).sum(1)
    return math.sqrt(sigma2) * math.sqrt(2.0 / K) * b


def responses(mu: np.ndarray, lik: int, rng, xi: float = 1.0) -> np.ndarray:
    if lik == LIK_BERNOULLI_LOGIT:
        p = 1.0 / (1.0 + np.exp(-mu))
        return (rng.random(len(mu)) < p).astype(np.float64)
    if lik == LIK_GAMMA_LOG:
        # shape xi, rate xi e^{-mu} (numpy takes the scale = 1 / rate): mean e^mu
        return rng.gamma(xi, np.exp(mu) / xi).astype(np.float64)
    return rng.poisson(np.exp(mu)).astype(np.float64)


def intercept_and_coords(locs: np.ndarray) -> np.ndarray:
    """Predictors of the linear term F = X beta used in Section 5: an intercept and the
    two coordinates, centred."""
    return np.column_stack([np.ones(len(locs)), locs - locs.mean(0) if len(locs) else locs])


def grid_with_gaps(nx: int, ny: int, remove: int, rng) -> np.ndarray:
    """Points ((i+1/2)/nx, (j+1/2)/ny) of an nx-by-ny grid over the unit square with
    axis-aligned rectangles (sides uniform in [0.01, 0.15], centres uniform) cut out
    until exactly ``remove`` points are gone; the last rectangle is trimmed in
    grid-index order."""
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    pts = np.stack([(ii.ravel() + 0.5) / nx, (jj.ravel() + 0.5) / ny], axis=1)
    keep = np.ones(len(pts), bool)
    removed = 0
    while removed < remove:
        w, h = rng.uniform(0.01, 0.15, size=2)
        cx, cy = rng.uniform(0.0, 1.0, size=2)
        # candidate grid block (one cell of slack), then the exact membership test
        i0, i1 = max(0, int((cx - w / 2) * nx) - 1), min(nx, int((cx + w / 2) * nx) + 2)
        j0, j1 = max(0, int((cy - h / 2) * ny) - 1), min(ny, int((cy + h / 2) * ny) + 2)
        cand = (np.arange(i0, i1)[:, None] * ny + np.arange(j0, j1)[None, :]).ravel()
        inside = keep[cand] & (np.abs(pts[cand, 0] - cx) <= w / 2) & (np.abs(pts[cand, 1] - cy) <= h / 2)
        idx = cand[inside]
        take = idx[: remove - removed]
        keep[take] = False
        removed += len(take)
    return pts[keep]


def make_problem(name: str, seed: int = 1, n: int | None = None) -> Problem:
    """Build a named workload. ``n`` overrides the size of the uniform workloads
    (used for smaller parity cases with the same recipe)."""
    rng = np.random.default_rng(seed)
    if name == "c1_n2000":
        nn = n or 2000
        locs = rng.random((nn, 2))
        cov, sigma2, rho, m, lik = COV_EXPONENTIAL, 1.0, 0.1, 10, LIK_BERNOULLI_LOGIT
        b = latent_exact(locs, cov, sigma2, rho, rng) if nn <= 6000 else latent_rff(locs, cov, sigma2, rho, rng)
        F = np.zeros(nn)
        test = rng.random((max(nn // 10, 1), 2))
        t, s = 50, 100
    elif name == "c2_n100k":
        nn = n or 100_000
        locs = rng.random((nn, 2))
        cov, sigma2, rho, m, lik = COV_MATERN15, 1.0, 0.05, 20, LIK_BERNOULLI_LOGIT
        b = latent_rff(locs, cov, sigma2, rho, rng)
        F = np.zeros(nn)
        test = rng.random((max(nn // 10, 1), 2))
        t, s = 50, 100
    elif name in ("c3_grid1m", "c3_grid800k"):
        if name == "c3_grid1m":
            nx, ny, rem = 1250, 1000, 250_000
        else:
            nx, ny, rem = 1000, 1000, 200_000
        if n is not None:  # same recipe on a smaller grid with the same 20% cut
            side = int(round(math.sqrt(n / 0.8)))
            nx, ny, rem = side, side, side * side - n
        locs = grid_with_gaps(nx, ny, rem, rng)
        cov, sigma2, rho, m, lik = COV_MATERN15, 1.0, 0.02, 20, LIK_POISSON_LOG
        b = latent_rff(locs, cov, sigma2, rho, rng)
        F = np.ones(len(locs))
        test = rng.random((1000, 2))
        t, s = 50, 100
    else:
        raise ValueError(f"unknown workload {name!r}")
    nn = len(locs)
    order = rng.permutation(nn).astype(np.int32)
    y = responses(F + b, lik, rng)
    Fp = np.full(len(test), F[0] if nn else 0.0)
    return Problem(name=name, locs=np.ascontiguousarray(locs), order=order, y=y, F=F, cov=cov,
                   sigma2=sigma2, rho=rho, m=m, lik=lik, t=t, s=s,
                   test_locs=np.ascontiguousarray(test), Fp=Fp, b_true=b, seed=seed)


def tiny_problem(n: int, m: int, cov: int = COV_MATERN15, lik: int = LIK_BERNOULLI_LOGIT,
                 rho: float = 0.2, sigma2: float = 1.0, seed: int = 3, n_test: int = 7,
                 F0: float = 0.0, xi: float = 1.0, beta=None) -> Problem:
    """Small uniform problem with an exact latent draw, for pins and edge cases. With
    ``beta`` the offset is F = X beta, X = intercept_and_coords(locs) (F0 is then unused)."""
    rng = np.random.default_rng(seed)
    locs = rng.random((n, 2))
    b = latent_exact(locs, cov, sigma2, rho, rng) if n > 0 else np.zeros(0)
    X = None
    if beta is None:
        F, Fp = np.full(n, F0), np.full(n_test, F0)
    else:
        beta = np.asarray(beta, float)
        X = intercept_and_coords(locs)
        F = X @ beta
    y = responses(F + b, lik, rng, xi)
    order = rng.permutation(n).astype(np.int32)
    test = rng.random((n_test, 2))
    if beta is not None:
        Fp = np.column_stack([np.ones(n_test), test - locs.mean(0)]) @ beta
    return Problem(name=f"tiny_n{n}_m{m}", locs=locs, order=order, y=y, F=F, cov=cov, sigma2=sigma2,
                   rho=rho, m=m, lik=lik, t=8, s=16, test_locs=test, Fp=Fp,
                   b_true=b, seed=seed, xi=xi, X=X, beta=beta)


def serving_params(rng) -> tuple[int, float, int]:
    """(n, range, likelihood) of one serving request, drawn first from its generator."""
    n = int(round(math.exp(rng.uniform(math.log(1e3), math.log(2e5)))))
    rho = float(rng.uniform(0.02, 0.2))
    lik = LIK_BERNOULLI_LOGIT if rng.random() < 0.5 else LIK_POISSON_LOG
    return n, rho, lik


def batched_params(rng) -> tuple[int, int, float]:
    """(n, m, range) of one problem of the batched workload, drawn first from its generator."""
    n = int(round(math.exp(rng.uniform(math.log(5e3), math.log(5e4)))))
    m = int(rng.choice([10, 20, 30]))
    rho = float(rng.uniform(0.02, 0.2))
    return n, m, rho


def serving_problem(index: int, seed: int = 7, n: int | None = None) -> Problem:
    """Request ``index`` of the serving stream: a fresh latent-GP problem with n
    log-uniform in [1e3, 2e5], uniform locations, Matern-1.5 covariance (sigma^2 = 1)
    with range uniform in [0.02, 0.2], m = 20, Bernoulli-logit or Poisson-log
    responses with probability 1/2 each, and 1000 uniform test points (t = 50 probes,
    s = 100 simulation vectors). The latent field uses 64 random Fourier features so
    that a stream of thousands of requests can be drawn in seconds."""
    rng = np.random.default_rng([seed, index])
    n0, rho, lik = serving_params(rng)
    nn = n or n0
    locs = rng.random((nn, 2))
    b = latent_rff(locs, COV_MATERN15, 1.0, rho, rng, K=64)
    F = np.zeros(nn)
    y = responses(F + b, lik, rng)
    order = rng.permutation(nn).astype(np.int32)
    test = rng.random((1000, 2))
    return Problem(name=f"serve_{index}", locs=locs, order=order, y=y, F=F, cov=COV_MATERN15, sigma2=1.0,
                   rho=rho, m=20, lik=lik, t=50, s=100, test_locs=test, Fp=np.zeros(1000), b_true=b,
                   seed=seed)


def batched_problem(index: int, seed: int = 5, n: int | None = None) -> Problem:
    """Problem ``index`` of the batched workload: n log-uniform in [5e3, 5e4], m
    uniform in {10, 20, 30}, uniform locations, exponential covariance (sigma^2 = 1)
    with range uniform in [0.02, 0.2], Bernoulli-logit responses, t = 50 probes."""
    rng = np.random.default_rng([seed, index])
    n0, m, rho = batched_params(rng)
    nn = n or n0
    locs = rng.random((nn, 2))
    b = latent_rff(locs, COV_EXPONENTIAL, 1.0, rho, rng, K=64)
    F = np.zeros(nn)
    y = responses(F + b, LIK_BERNOULLI_LOGIT, rng)
    order = rng.permutation(nn).astype(np.int32)
    return Problem(name=f"batch_{index}", locs=locs, order=order, y=y, F=F, cov=COV_EXPONENTIAL, sigma2=1.0,
                   rho=rho, m=m, lik=LIK_BERNOULLI_LOGIT, t=50, s=100, test_locs=None, Fp=None, b_true=b,
                   seed=seed)


def poisson_arrivals(rate: float, duration: float, seed: int = 11) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate on [0, duration)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return np.array(out)
        out.append(t)
