"""The L-BFGS estimation loop (paper_2310_12000_gb300/estimate.py) driven by the oracle's
exact L^VLA and gradient on CPU: it reaches a stationary point, from different starts the
same one, and the minimum is below its neighbours."""
import numpy as np

import workloads as wl
from oracle import gradients as gr, laplace as la
from paper_2310_12000_gb300 import estimate


def _oracle_objective(P):
    base = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)

    def obj(theta):
        f = la.refit(base, float(theta[0]), float(theta[1]), 1e-10 * float(theta[0]))
        md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-12)
        L, _ = la.lml_exact(f, md)
        g = gr.lml_grad_exact(f, md)
        return L, np.array([g["sigma2"], g["rho"]])
    return obj


def test_lbfgs_finds_the_same_stationary_point_from_two_starts():
    P = wl.tiny_problem(150, 10, lik=wl.LIK_POISSON_LOG, rho=0.2, sigma2=1.0, F0=0.5)
    obj = _oracle_objective(P)
    r1 = estimate.fit(obj, [0.5, 0.1], max_iter=60)
    r2 = estimate.fit(obj, [2.0, 0.4], max_iter=60)
    assert r1.converged and r2.converged, (r1.message, r2.message)
    assert np.allclose(r1.theta, r2.theta, rtol=1e-3)
    # stationary in log space and a local minimum along each axis
    assert np.max(np.abs(r1.grad * r1.theta)) < 1e-3
    for k in range(2):
        for s in (0.97, 1.03):
            th = r1.theta.copy()
            th[k] *= s
            assert obj(th)[0] >= r1.value - 1e-9


class _OracleState:
    def __init__(self, f, md):
        self.f, self.md = f, md

    def log_marglik(self, opts):
        return la.lml_exact(self.f, self.md)[0]

    def lml_grad(self, opts, offset=False):
        g = gr.lml_grad_exact(self.f, self.md)
        g = np.array([g["sigma2"], g["rho"]])
        return (g, gr.lml_grad_F_exact(self.f, self.md)) if offset else g

    def close(self):
        pass


class _OracleFactor:
    """The three factor calls library_objective makes, answered by the exact oracle."""

    def __init__(self, P):
        self.P = P
        self.f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)

    def refit(self, s2, rho, opts):
        self.f = la.refit(self.f, s2, rho, 1e-10 * s2)

    def find_mode(self, lik, y, F, opts):
        return _OracleState(self.f, la.find_mode(self.f, y, F, lik, newton_tol=1e-12, xi=self.P.xi))


def test_library_objective_with_predictors_chains_the_offset_gradient():
    """With X the objective's offset is X beta and its beta-gradient X^T dL/dF: checked against
    central differences of the exact L^VLA in beta (and the covariance part unchanged)."""
    P = wl.tiny_problem(120, 9, lik=wl.LIK_POISSON_LOG, rho=0.2, beta=[0.4, -0.5, 0.3])
    obj = estimate.library_objective(None, _OracleFactor(P), P.lik, P.y, None, None, X=P.X)
    theta = np.array([0.9, 0.17, 0.35, -0.45, 0.2])
    L, g = obj(theta)
    assert g.shape == (5,)
    h = 1e-5
    for k in range(5):
        e = np.zeros(5)
        e[k] = h
        fd = (obj(theta + e)[0] - obj(theta - e)[0]) / (2 * h)
        assert abs(g[k] - fd) < 1e-5 * (1 + abs(fd)), (k, g[k], fd)
    # an offset F adds to X beta
    obj2 = estimate.library_objective(None, _OracleFactor(P), P.lik, P.y, np.full(P.n, 0.1), None, X=P.X)
    th2 = theta.copy()
    th2[2] -= 0.1                          # intercept absorbs the constant offset
    assert abs(obj2(th2)[0] - L) < 1e-9 * abs(L)


def test_joint_fit_of_covariance_and_coefficients():
    P = wl.tiny_problem(140, 10, lik=wl.LIK_POISSON_LOG, rho=0.2, seed=4, beta=[0.5, 0.8, -0.6])
    obj = estimate.library_objective(None, _OracleFactor(P), P.lik, P.y, None, None, X=P.X)
    r1 = estimate.fit(obj, [0.6, 0.1, 0.0, 0.0, 0.0], max_iter=100, n_positive=2)
    r2 = estimate.fit(obj, [1.6, 0.3, 1.0, 0.0, 0.0], max_iter=100, n_positive=2)
    assert r1.converged and r2.converged, (r1.message, r2.message)
    assert np.allclose(r1.theta, r2.theta, rtol=2e-3, atol=2e-3)
    scale = np.concatenate([r1.theta[:2], np.ones(3)])
    assert np.max(np.abs(r1.grad * scale)) < 1e-3
    for k in range(5):
        for s in (-1, 1):
            th = r1.theta.copy()
            th[k] = th[k] * (1 + 0.03 * s) if k < 2 else th[k] + 0.03 * s
            assert obj(th)[0] >= r1.value - 1e-9


def test_fit_rejects_mismatched_bounds():
    import pytest
    with pytest.raises(ValueError):
        estimate.fit(lambda th: (0.0, np.zeros(3)), [1.0, 0.1, 0.0], bounds=[(1e-3, 1e3)], n_positive=2)


def test_joint_fit_with_the_gamma_shape():
    """Section 5's parameter set: covariance (sigma2, range), the gamma shape alpha (all
    positive, searched in log space) and the coefficients beta, on the oracle's exact L^VLA
    and gradient. The fit reaches a stationary point and a local minimum."""
    P = wl.tiny_problem(120, 8, lik=wl.LIK_GAMMA_LOG, rho=0.2, sigma2=0.5, seed=6, xi=5.0, beta=[0.3, 0.4, -0.2])
    base = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)

    def obj(theta):
        s2, rho, a = (float(v) for v in theta[:3])
        f = la.refit(base, s2, rho, 1e-10 * s2)
        F = P.X @ theta[3:]
        md = la.find_mode(f, P.y, F, la.LIK_GAMMA_LOG, newton_tol=1e-12, xi=a)
        L, _ = la.lml_exact(f, md)
        g = gr.lml_grad_exact(f, md)
        dF = gr.lml_grad_F_exact(f, md)
        return L, np.concatenate([[g["sigma2"], g["rho"], gr.lml_grad_xi_exact(f, md)], gr.lml_grad_beta(P.X, dF)])

    bounds = [(1e-3, 1e3), (1e-3, 10.0), (1e-2, 1e4), (None, None), (None, None), (None, None)]
    r = estimate.fit(obj, [1.0, 0.1, 2.0, 0.0, 0.0, 0.0], max_iter=200, n_positive=3, bounds=bounds)
    assert r.converged, r.message
    scale = np.concatenate([r.theta[:3], np.ones(3)])
    assert np.max(np.abs(r.grad * scale)) < 1e-3
    for k in range(6):
        for s in (-1, 1):
            th = r.theta.copy()
            th[k] = th[k] * (1 + 0.03 * s) if k < 3 else th[k] + 0.03 * s
            assert obj(th)[0] >= r.value - 1e-9
