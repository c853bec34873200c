"""Gamma likelihood (Section 5: y | mu ~ Gamma(a, a e^{-mu}), E[y | mu] = e^mu) with the
linear term F = X beta, through the C ABI against the oracle on the same seeded inputs and
probes: mode, L^VLA, every SLQ term and the predictive mean and variances within 1e-9 in
float64, and within 1e-4 in mixed precision; a shape <= 0 and the gradient (Bernoulli and
Poisson only) are refused. The newest GPU tests, so they run last."""
import numpy as np
import pytest

import workloads as wl
from oracle import laplace as la

pytestmark = pytest.mark.gpu

FP64_TIGHT = dict(cg_tol=1e-12, newton_tol=1e-10, cg_max_iter=2000)


def _problem():
    return wl.tiny_problem(600, 10, lik=wl.LIK_GAMMA_LOG, rho=0.15, sigma2=0.5, seed=12, n_test=40, xi=6.0,
                           beta=[0.4, 0.5, -0.3])


def _oracle(P):
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, la.LIK_GAMMA_LOG, newton_tol=1e-10, xi=P.xi)
    return f, md


def test_gamma_parity_fp64_and_mixed():
    import paper_2310_12000_gb300 as vl
    vl.library()
    P = _problem()
    ctx = vl.Context(0, ws_bytes=1 << 30)
    t, s = 16, 32
    o64 = vl.Opts.make(t=t, s=s, lik_shape=P.xi, **FP64_TIGHT)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, o64)
    st = fac.find_mode(vl.LIK_GAMMA_LOG, P.y, P.F, o64)
    lml = st.log_marglik(o64)
    gam = st.slq_gammas(t)
    mean, var = st.pred_var(P.test_locs, P.Fp, o64)

    f, md = _oracle(P)
    b_ref = la.mode_user(f, md)
    assert np.max(np.abs(st.mode - b_ref)) / np.max(np.abs(b_ref)) < 1e-9
    L_ref, _, g_ref = la.lml_slq(f, md, t, 1)
    assert np.max(np.abs(gam - g_ref) / np.maximum(np.abs(g_ref), 1.0)) < 1e-9
    assert abs(lml - L_ref) / abs(L_ref) < 1e-9
    pf = la.pred_factor(f, P.test_locs, P.m)
    assert np.max(np.abs(mean - la.pred_mean(pf, md, P.Fp))) < 1e-9 * (1 + np.max(np.abs(mean)))
    v_ref = la.pred_var_sim(f, md, pf, s, 1)
    assert np.max(np.abs(var - v_ref) / v_ref) < 1e-9

    o32 = vl.Opts.make(t=t, precision=vl.FP32_REFINE, cg_tol=1e-6, newton_tol=1e-7, lik_shape=P.xi)
    st32 = fac.find_mode(vl.LIK_GAMMA_LOG, P.y, P.F, o32)
    lml32 = st32.log_marglik(o32)
    assert abs(lml32 - L_ref) / abs(L_ref) < 1e-4
    assert np.max(np.abs(st32.mode - b_ref)) / np.max(np.abs(b_ref)) < 1e-4
    st32.close()
    st.close()
    ctx.close()


def test_gamma_refusals():
    import paper_2310_12000_gb300 as vl
    P = _problem()
    ctx = vl.Context(0, ws_bytes=256 << 20)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    for a in (0.0, -1.0, float("nan")):
        with pytest.raises(vl.VLError):
            fac.find_mode(vl.LIK_GAMMA_LOG, P.y, P.F, vl.Opts.make(lik_shape=a))
    # a response outside the gamma support (y <= 0, or not finite) is refused before Newton,
    # naming its caller index
    for bad in (0.0, -2.0, float("inf")):
        y = P.y.copy()
        y[5] = bad
        with pytest.raises(vl.VLError) as e:
            fac.find_mode(vl.LIK_GAMMA_LOG, y, P.F, vl.Opts.make(lik_shape=P.xi))
        assert e.value.status == 1 and "y[5]" in str(e.value), str(e.value)
    st = fac.find_mode(vl.LIK_GAMMA_LOG, P.y, P.F, vl.Opts.make(lik_shape=P.xi, **FP64_TIGHT))
    with pytest.raises(vl.VLError):
        st.lml_grad(vl.Opts.make(t=8, lik_shape=P.xi))
    st.close()
    ctx.close()
