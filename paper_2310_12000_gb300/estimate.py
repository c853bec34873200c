"""Covariance-parameter estimation by L-BFGS on the Vecchia-Laplace negative log-marginal
likelihood (Section 4: L-BFGS with a sample average approximation).

The objective at theta = (sigma2, range) is L^VLA (Eq. VLA_loss) with its gradient; with the
stochastic log-determinant (SLQ, Eq. def_SLQ) and its gradient (STE, Eq. grad_STE) the probes
are fixed across iterations (the same seed every evaluation), which is the sample average
approximation: the optimiser sees one deterministic function. The search runs over
log-parameters so both stay positive.

``fit`` takes any objective theta -> (L, dL/dtheta); ``library_objective`` builds it from the
library calls on one factor: refit (Section 2.1), mode (Eq. newton), L^VLA and its gradient.
"""
from __future__ import annotations

import dataclasses
from typing import Callable

import numpy as np


@dataclasses.dataclass
class FitResult:
    theta: np.ndarray          # (sigma2, range)
    value: float               # L^VLA at theta
    grad: np.ndarray           # dL/dtheta at theta
    evaluations: int
    converged: bool
    message: str


def fit(objective: Callable[[np.ndarray], tuple[float, np.ndarray]], theta0, max_iter: int = 50,
        gtol: float = 1e-5, bounds=((1e-3, 1e3), (1e-4, 10.0))) -> FitResult:
    """Minimises objective(theta) over theta = (sigma2, range) with L-BFGS-B in log space."""
    from scipy.optimize import minimize

    calls = {"n": 0}
    cache = {}

    def f(u):
        theta = np.exp(u)
        L, g = objective(theta)
        calls["n"] += 1
        cache["last"] = (theta, L, np.asarray(g, float))
        return float(L), np.asarray(g, float) * theta     # d/du = theta * d/dtheta

    lb = [(np.log(lo), np.log(hi)) for lo, hi in bounds]
    res = minimize(f, np.log(np.asarray(theta0, float)), jac=True, method="L-BFGS-B", bounds=lb,
                   options={"maxiter": max_iter, "gtol": gtol})
    theta = np.exp(res.x)
    L, g = objective(theta)
    return FitResult(theta=theta, value=float(L), grad=np.asarray(g, float), evaluations=calls["n"] + 1,
                     converged=bool(res.success), message=str(res.message))


def library_objective(vl, fac, lik: int, y, F, opts) -> Callable[[np.ndarray], tuple[float, np.ndarray]]:
    """theta -> (L^VLA, (dL/dsigma2, dL/drange)) through the library on factor `fac` (its
    neighbours and level schedules are reused; only A_i, D_i are recomputed). opts fixes the
    probes (seed, t) for every evaluation; the gradient needs float64 with VADU."""
    def obj(theta):
        fac.refit(float(theta[0]), float(theta[1]), opts)
        st = fac.find_mode(lik, y, F, opts)
        try:
            L = st.log_marglik(opts)
            g = st.lml_grad(opts)
        finally:
            st.close()
        return L, g
    return obj
