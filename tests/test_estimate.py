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
