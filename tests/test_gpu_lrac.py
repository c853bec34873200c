"""LRAC preconditioner (Section 3.1.2, Eqs. P_LRAC, pcls2, logdetsplit2) on the CUDA
path vs the CPU oracle, through the C ABI, on the same seeded inputs.

Pivots are integer decisions taken in float64 on both sides: they must agree
exactly on inputs without exact distance ties (uniform random locations). With
equal pivots the float64 path is held to 1e-9 relative like the other
preconditioners; the mixed-precision path to 1e-4 on L^VLA and 1e-6 on the
float64 residual of every refined solve.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import laplace as la, lrac as olr

pytestmark = pytest.mark.gpu

FP64_TIGHT = dict(cg_tol=1e-12, newton_tol=1e-10, cg_max_iter=3000)


@pytest.fixture(scope="module")
def vl():
    import paper_2310_12000_gb300 as vl
    vl.library()
    return vl


@pytest.fixture(scope="module")
def ctx(vl):
    return vl.Context(0, ws_bytes=4 << 30)


def _oracle_all(P, newton_tol=1e-10):
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=newton_tol)
    return f, md


def _lrac(vl, **kw):
    return vl.Opts.make(precond=vl.PREC_LRAC, **kw)


# ----------------------------------------------------------------------------- pivoted Cholesky
@pytest.mark.parametrize("name,n,k", [("c1_n2000", 1500, 1), ("c1_n2000", 1500, 37), ("c2_n100k", 2000, 64),
                                      ("c2_n100k", 2000, 130)])
def test_pivoted_cholesky_parity(ctx, vl, name, n, k):
    P = wl.make_problem(name, n=n)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    piv, L = fac.lrac_export(k)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    L_ref, piv_ref = olr.pivoted_cholesky(f.locs, f.cov, f.sigma2, f.rho, f.nugget, k)
    assert np.array_equal(piv, piv_ref)
    assert np.max(np.abs(L[f.order] - L_ref)) < 1e-9


def test_pivoted_cholesky_rebuilt_after_refit(ctx, vl):
    P = wl.make_problem("c1_n2000", n=800)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    _, L1 = fac.lrac_export(20)
    fac.refit(2.0, 0.05)
    _, L2 = fac.lrac_export(20)
    f = la.build_factor(P.locs, P.order, P.cov, 2.0, 0.05, P.m, 1e-10 * 2.0)
    L_ref, _ = olr.pivoted_cholesky(f.locs, f.cov, 2.0, 0.05, f.nugget, 20)
    assert np.max(np.abs(L2[f.order] - L_ref)) < 1e-9
    assert np.max(np.abs(L1 - L2)) > 1e-3


def test_lrac_rank_errors(ctx, vl):
    P = wl.tiny_problem(40, 10)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    with pytest.raises(vl.VLError):
        fac.lrac_export(41)          # k > n
    with pytest.raises(vl.VLError):
        fac.find_mode(P.lik, P.y, P.F, _lrac(vl, k=0))
    with pytest.raises(vl.VLError):
        fac.find_mode(P.lik, P.y, P.F, _lrac(vl, k=1025))
    piv, L = fac.lrac_export(40)     # k = n is allowed
    assert sorted(piv.tolist()) == list(range(40))


# ----------------------------------------------------------------------------- operators
@pytest.mark.parametrize("t", [1, 5, 70])
def test_woodbury_apply_and_form2_solve(ctx, vl, t):
    P = wl.make_problem("c1_n2000", n=500)
    k = 40
    opts = _lrac(vl, k=k, **FP64_TIGHT)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts)
    st = fac.find_mode(P.lik, P.y, P.F, opts)
    f, md = _oracle_all(P)
    L_ref, _ = olr.pivoted_cholesky(f.locs, f.cov, f.sigma2, f.rho, f.nugget, k)
    X = np.random.default_rng(t).standard_normal((P.n, t))
    Y = st.apply(vl.OP_PINV, X, opts)
    Yv = olr.woodbury_apply(L_ref, md.W, X[f.order])
    assert np.max(np.abs(Y[f.order] - Yv)) < 1e-10 * np.max(np.abs(Yv))
    # the form-2 system (Sigma_tilde + W^{-1}) U = R
    A2 = olr.sigma_tilde_dense(f) + np.diag(1.0 / md.W)
    U, _, _, it, rel = st.pcg_solve(X, opts)
    Uv = np.linalg.solve(A2, X[f.order])
    assert np.max(np.abs(U[f.order] - Uv)) < 1e-9 * np.max(np.abs(Uv))
    assert np.all(rel <= 1e-12)


# ----------------------------------------------------------------------------- L^VLA
@pytest.mark.parametrize("t,k", [(1, 20), (16, 50), (70, 33)])
def test_lrac_mode_and_lml_parity_fp64(ctx, vl, t, k):
    P = wl.make_problem("c1_n2000", n=600)
    opts = _lrac(vl, t=t, k=k, **FP64_TIGHT)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts)
    st = fac.find_mode(P.lik, P.y, P.F, opts)
    lml, stats = st.log_marglik(opts, with_stats=True)
    f, md = _oracle_all(P)
    piv, _ = fac.lrac_export(k, with_L=False)
    _, piv_ref = olr.pivoted_cholesky(f.locs, f.cov, f.sigma2, f.rho, f.nugget, k)
    assert np.array_equal(piv, piv_ref)
    b_ref = la.mode_user(f, md)
    assert np.max(np.abs(st.mode - b_ref)) / np.max(np.abs(b_ref)) < 1e-9
    L_ref, ld_ref, g_ref = olr.lml_lrac_dense(f, md, k, t, 1)
    g = st.slq_gammas(t)
    assert np.max(np.abs(g - g_ref) / np.maximum(np.abs(g_ref), 1.0)) < 1e-9
    assert abs(lml - L_ref) / abs(L_ref) < 1e-9
    assert abs(stats["logdet"] - ld_ref) < 1e-9 * max(1.0, abs(ld_ref))


def test_lrac_full_rank_is_exact(ctx, vl):
    """m = n-1 and k = n: P_LRAC = Sigma + W^{-1} is the form-2 matrix itself, so
    every probe solve stops after one step and log det(I + L^T W L) alone is the
    exact log-determinant."""
    P = wl.tiny_problem(60, 59, rho=0.3)
    opts = _lrac(vl, t=8, k=60, **FP64_TIGHT)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts)
    st = fac.find_mode(P.lik, P.y, P.F, opts)
    lml, stats = st.log_marglik(opts, with_stats=True)
    f, md = _oracle_all(P)
    L_ex, ld_ex = la.lml_exact(f, md)
    assert stats["cg_iters_max"] <= 2
    assert abs(stats["slq_mean"]) < 1e-8 * abs(ld_ex)
    assert abs(lml - L_ex) < 1e-8 * abs(L_ex)


def test_lrac_pred_var_parity_fp64(ctx, vl):
    P = wl.make_problem("c1_n2000", n=700)
    P.test_locs = P.test_locs[:200]
    opts = _lrac(vl, k=30, s=40, **FP64_TIGHT)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts)
    st = fac.find_mode(P.lik, P.y, P.F, opts)
    mean, var = st.pred_var(P.test_locs, None, opts)
    f, md = _oracle_all(P)
    pf = la.pred_factor(f, P.test_locs, P.m)
    v_ref = la.pred_var_sim(f, md, pf, 40, 1)
    assert np.max(np.abs(var - v_ref) / v_ref) < 1e-9


def test_lrac_mixed_precision(ctx, vl):
    P = wl.make_problem("c1_n2000")
    k, t = 50, 30
    o64 = _lrac(vl, t=t, k=k, **FP64_TIGHT)
    o32 = _lrac(vl, t=t, k=k, precision=vl.FP32_REFINE, cg_tol=1e-6, newton_tol=1e-7)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, o64)
    st32 = fac.find_mode(P.lik, P.y, P.F, o32)
    ms = st32.mode_stats()
    assert ms["true_relres_max"] <= 1e-6
    lml32 = st32.log_marglik(o32)
    f, md = _oracle_all(P)
    piv, _ = fac.lrac_export(k, with_L=False)
    _, piv_ref = olr.pivoted_cholesky(f.locs, f.cov, f.sigma2, f.rho, f.nugget, k)
    assert np.array_equal(piv, piv_ref)
    L_ref, _, _ = olr.lml_lrac_dense(f, md, k, t, 1)
    assert abs(lml32 - L_ref) / abs(L_ref) < 1e-4
    b_ref = la.mode_user(f, md)
    assert np.max(np.abs(st32.mode - b_ref)) / np.max(np.abs(b_ref)) < 1e-4
    o32p = _lrac(vl, k=k, s=32, precision=vl.FP32_REFINE, cg_tol=1e-6)
    _, var, vs = st32.pred_var(P.test_locs[:300], None, o32p, with_stats=True)
    assert vs["true_relres_max"] <= 1e-6
    pf = la.pred_factor(f, P.test_locs[:300], P.m)
    v_ref = la.pred_var_sim(f, md, pf, 32, 1)
    assert np.max(np.abs(var - v_ref) / v_ref) < 1e-4


def test_lrac_poisson_grid_consistent_with_exact(ctx, vl):
    """Satellite-swath grid (exact distance ties, so pivots may legitimately differ
    from the oracle's at the rounding level): the LRAC estimate must agree with the
    exact Laplace value within the SLQ's own standard error, and with the VADU run."""
    P = wl.make_problem("c3_grid1m", n=3000)
    o = _lrac(vl, t=50, k=100, precision=vl.FP32_REFINE, cg_tol=1e-6, newton_tol=1e-7)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, o)
    st = fac.find_mode(P.lik, P.y, P.F, o)
    lml, stats = st.log_marglik(o, with_stats=True)
    f, md = _oracle_all(P)
    L_ex, _ = la.lml_exact(f, md)
    assert abs(lml - L_ex) < 4 * 0.5 * stats["slq_stderr"] + 1e-4 * abs(L_ex)


# ----------------------------------------------------------------------------- tensor-core products
@pytest.mark.parametrize("n,k,t", [(1037, 37, 2), (1037, 130, 7), (2000, 500, 50), (1500, 64, 64), (777, 200, 1)])
def test_woodbury_apply_float32_tensor_cores(ctx, vl, n, k, t):
    """Float32 blocks of 2..64 columns take the tcgen05 (tf32, split-operand) products;
    t = 1 the SIMT ones. Both must agree with the float64 Woodbury identity to
    float32 accuracy."""
    P = wl.make_problem("c1_n2000", n=n)
    o64 = _lrac(vl, k=k, **FP64_TIGHT)
    o32 = _lrac(vl, k=k, precision=vl.FP32_REFINE, cg_tol=1e-6, newton_tol=1e-7)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, o64)
    st = fac.find_mode(P.lik, P.y, P.F, o64)
    f, md = _oracle_all(P)
    L_ref, _ = olr.pivoted_cholesky(f.locs, f.cov, f.sigma2, f.rho, f.nugget, k)
    X = np.random.default_rng(n + t).standard_normal((P.n, t))
    Y = st.apply(vl.OP_PINV, X, o32)
    Yv = olr.woodbury_apply(L_ref, md.W, X[f.order])
    err = np.max(np.abs(Y[f.order] - Yv)) / np.max(np.abs(Yv))
    assert err < 2e-5, err
