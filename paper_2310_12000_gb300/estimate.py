"""Covariance-parameter estimation by L-BFGS on the Vecchia-Laplace negative log-marginal
likelihood (Section 4: L-BFGS with a sample average approximation).

The objective at theta = (sigma2, range) is L^VLA (Eq. VLA_loss) with its gradient; with the
stochastic log-determinant (SLQ, Eq. def_SLQ) and its gradient (STE, Eq. grad_STE) the probes
are fixed across iterations (the same seed every evaluation), which is the sample average
approximation: the optimiser sees one deterministic function. The search runs over
log-parameters so both stay positive.

``fit`` takes any objective theta -> (L, dL/dtheta); ``library_objective`` builds it from the
library calls on one factor: refit (Section 2.1), mode (Eq. newton), L^VLA and its gradient.
With predictors X the offset is the linear term F = X beta (Section 2) and theta carries the
coefficients after (sigma2, range); their gradient is dL/dbeta = X^T dL/dF, from the same
probe solves as the covariance gradient.
"""
from __future__ import annotations

import dataclasses
from typing import Callable

import numpy as np


COV_BOUNDS = ((1e-3, 1e3), (1e-4, 10.0))      # sigma2, range


@dataclasses.dataclass
class FitResult:
    theta: np.ndarray          # (sigma2, range[, beta...])
    value: float               # L^VLA at theta
    grad: np.ndarray           # dL/dtheta at theta
    evaluations: int
    converged: bool
    message: str


def fit(objective: Callable[[np.ndarray], tuple[float, np.ndarray]], theta0, max_iter: int = 50,
        gtol: float = 1e-5, bounds=None, n_positive: int | None = None) -> FitResult:
    """Minimises objective(theta) with L-BFGS-B. The first n_positive entries of theta (all of
    them by default) are positive and searched in log space; the rest (coefficients beta) as
    they are. bounds, one (lo, hi) per entry in natural units (None = open), defaults to
    COV_BOUNDS for (sigma2, range) and open bounds after them."""
    from scipy.optimize import minimize

    theta0 = np.asarray(theta0, float)
    k = len(theta0)
    npos = k if n_positive is None else int(n_positive)
    if bounds is None:
        bounds = list(COV_BOUNDS[:min(2, npos)]) + [(None, None)] * (k - min(2, npos))
    if len(bounds) != k or not 0 <= npos <= k:
        raise ValueError("one bound per parameter and 0 <= n_positive <= len(theta0)")
    calls = {"n": 0}

    def to_theta(u):
        return np.concatenate([np.exp(u[:npos]), u[npos:]])

    def f(u):
        theta = to_theta(u)
        L, g = objective(theta)
        calls["n"] += 1
        g = np.asarray(g, float).copy()
        g[:npos] *= theta[:npos]                         # d/du = theta * d/dtheta
        return float(L), g

    def log_bound(b):
        return None if b is None else float(np.log(b))

    ub = [(log_bound(lo), log_bound(hi)) if i < npos else (lo, hi) for i, (lo, hi) in enumerate(bounds)]
    u0 = np.concatenate([np.log(theta0[:npos]), theta0[npos:]])
    res = minimize(f, u0, jac=True, method="L-BFGS-B", bounds=ub, options={"maxiter": max_iter, "gtol": gtol})
    theta = to_theta(res.x)
    L, g = objective(theta)
    return FitResult(theta=theta, value=float(L), grad=np.asarray(g, float), evaluations=calls["n"] + 1,
                     converged=bool(res.success), message=str(res.message))


def library_objective(vl, fac, lik: int, y, F, opts, X=None) -> Callable[[np.ndarray], tuple[float, np.ndarray]]:
    """theta -> (L^VLA, dL/dtheta) through the library on factor `fac` (its neighbours and
    level schedules are reused; only A_i, D_i are recomputed), theta = (sigma2, range) or,
    with predictors X (n x p, caller order), (sigma2, range, beta_1..beta_p) and offset
    F + X beta (F may be None). opts fixes the probes (seed, t) for every evaluation; the
    gradient needs float64 with VADU."""
    Xm = None if X is None else np.ascontiguousarray(X, dtype=np.float64)
    F0 = None if F is None else np.asarray(F, np.float64)

    def obj(theta):
        theta = np.asarray(theta, float)
        fac.refit(float(theta[0]), float(theta[1]), opts)
        off = F0
        if Xm is not None:
            off = Xm @ theta[2:] if F0 is None else F0 + Xm @ theta[2:]
        st = fac.find_mode(lik, y, off, opts)
        try:
            L = st.log_marglik(opts)
            if Xm is None:
                return L, np.asarray(st.lml_grad(opts), float)
            g, dF = st.lml_grad(opts, offset=True)
        finally:
            st.close()
        return L, np.concatenate([np.asarray(g, float), Xm.T @ dF])
    return obj
