"""Gradient of L^VLA by stochastic trace estimation (Eq. grad_STE, control variate of
Section 3) on the CUDA path vs the oracle's same-probe estimate, float64, VADU."""
import numpy as np
import pytest

import workloads as wl
from oracle import gradients as gr, laplace as la

pytestmark = pytest.mark.gpu

FP64_TIGHT = dict(cg_tol=1e-12, newton_tol=1e-10, cg_max_iter=3000)


@pytest.mark.parametrize("name,n,t", [("c1_n2000", 500, 16), ("c3_grid1m", 800, 24)])
def test_lml_grad_matches_oracle_same_probes(name, n, t):
    import paper_2310_12000_gb300 as vl
    vl.library()
    ctx = vl.Context(0, ws_bytes=1 << 30)
    P = wl.make_problem(name, n=n)
    opts = vl.Opts.make(t=t, **FP64_TIGHT)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts)
    st = fac.find_mode(P.lik, P.y, P.F, opts)
    g, dF = st.lml_grad(opts, offset=True)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-12)
    ref = gr.lml_grad_ste(f, md, t, 1)["grad"]
    for k, par in enumerate(gr.PARAMS):
        assert abs(g[k] - ref[par]) < 1e-7 * (1.0 + abs(ref[par])), (par, g[k], ref[par])
    assert np.max(np.abs(dF - ref["F"])) < 1e-7 * (1.0 + np.max(np.abs(ref["F"])))
    ctx.close()


def test_lml_grad_rejects_unsupported_options():
    import paper_2310_12000_gb300 as vl
    ctx = vl.Context(0, ws_bytes=256 << 20)
    P = wl.tiny_problem(80, 8)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    st = fac.find_mode(P.lik, P.y, P.F, vl.Opts.make(**FP64_TIGHT))
    with pytest.raises(vl.VLError):
        st.lml_grad(vl.Opts.make(precision=vl.FP32_REFINE))
    with pytest.raises(vl.VLError):
        st.lml_grad(vl.Opts.make(precond=vl.PREC_LVA))
    ctx.close()
