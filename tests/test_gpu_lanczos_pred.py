"""Lanczos predictive variances (Section 4, preconditioner P_L1) on the GPU against the oracle
(oracle/lanczos_pred.py, float64, the same start vector and full reorthogonalisation): within
1e-9 relative at ranks k = 5, 20 and 60, and at k = n where both equal the exact variances
D_p + e_p^T B_po (W + Sigma_tilde^{-1})^{-1} B_po^T e_p; the mean is the one of vl_pred_var."""
import numpy as np
import pytest

import workloads as wl
from oracle import laplace as la
from oracle import lanczos_pred as lp

pytestmark = pytest.mark.gpu

FP64_TIGHT = dict(cg_tol=1e-12, newton_tol=1e-10, cg_max_iter=2000)


@pytest.fixture(scope="module")
def case():
    import paper_2310_12000_gb300 as vl
    vl.library()
    P = wl.tiny_problem(400, 10, rho=0.15, n_test=60, lik=wl.LIK_POISSON_LOG, F0=0.2, seed=12)
    ctx = vl.Context(0, ws_bytes=1 << 30)
    opts = vl.Opts.make(**FP64_TIGHT)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts)
    st = fac.find_mode(P.lik, P.y, P.F, opts)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-12)
    pf = la.pred_factor(f, P.test_locs, P.m)
    yield vl, P, st, f, md, pf
    ctx.close()


@pytest.mark.parametrize("k", [5, 20, 60])
def test_lanczos_variances_match_the_oracle(case, k):
    vl, P, st, f, md, pf = case
    mean, var, stats = st.pred_var_lanczos(P.test_locs, k, P.Fp, with_stats=True)
    ref = lp.pred_var_lanczos(f, md, pf, k, 1)
    assert stats["cg_iters_max"] == k
    assert np.max(np.abs(var - ref) / ref) < 1e-9, k
    assert np.max(np.abs(mean - la.pred_mean(pf, md, P.Fp))) < 1e-9 * (1 + np.max(np.abs(mean)))


def test_lanczos_variances_exact_at_full_rank(case):
    vl, P, st, f, md, pf = case
    _, var, stats = st.pred_var_lanczos(P.test_locs, P.n, P.Fp, with_stats=True)
    exact = la.pred_var_exact(f, md, pf)
    assert np.max(np.abs(var - exact) / exact) < 1e-8
    # and the error falls with the rank (the estimate is biased low for small k)
    errs = [np.max(np.abs(st.pred_var_lanczos(P.test_locs, k, P.Fp)[1] - exact)) for k in (5, 20, 60)]
    assert errs[2] <= errs[1] <= errs[0]


def test_lanczos_refusals(case):
    vl, P, st, f, md, pf = case
    with pytest.raises(vl.VLError):
        st.pred_var_lanczos(P.test_locs, 10, P.Fp, precond_l=2)
    with pytest.raises(vl.VLError):
        st.pred_var_lanczos(P.test_locs, 0, P.Fp)
