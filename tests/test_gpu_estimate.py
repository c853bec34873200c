"""The library objective of the estimation loop on the GPU: one evaluation equals the
oracle's same-probe L^VLA and STE gradient, and a short L-BFGS run reaches a stationary
point of the (fixed-probe) objective."""
import numpy as np
import pytest

import workloads as wl
from oracle import gradients as gr, laplace as la

pytestmark = pytest.mark.gpu


def test_library_objective_and_fit():
    import paper_2310_12000_gb300 as vl
    from paper_2310_12000_gb300 import estimate
    vl.library()
    ctx = vl.Context(0, ws_bytes=1 << 30)
    P = wl.make_problem("c1_n2000", n=400)
    opts = vl.Opts.make(t=16, cg_tol=1e-12, newton_tol=1e-10, cg_max_iter=3000)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts)
    obj = estimate.library_objective(vl, fac, P.lik, P.y, P.F, opts)
    theta = np.array([1.3, 0.08])
    L, g = obj(theta)
    f = la.build_factor(P.locs, P.order, P.cov, 1.3, 0.08, P.m, 1.3e-10)
    md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-12)
    L_ref, _, _ = la.lml_slq(f, md, 16, 1)
    g_ref = gr.lml_grad_ste(f, md, 16, 1)["grad"]
    assert abs(L - L_ref) < 1e-9 * abs(L_ref)
    assert abs(g[0] - g_ref["sigma2"]) < 1e-7 * (1 + abs(g_ref["sigma2"]))
    assert abs(g[1] - g_ref["rho"]) < 1e-7 * (1 + abs(g_ref["rho"]))
    r = estimate.fit(obj, [1.0, 0.1], max_iter=25)
    assert np.max(np.abs(r.grad * r.theta)) < 1e-2 * (1 + abs(r.value)) ** 0.5
    ctx.close()
