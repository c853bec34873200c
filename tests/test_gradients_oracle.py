"""Pins of the gradient oracle (oracle/gradients.py): every derivative against
central differences of the quantity it differentiates, and the stochastic trace
estimate against the exact derivative within its own standard error."""
import numpy as np
import pytest

import workloads as wl
from oracle import gradients as gr, laplace as la, vecchia


def _factor(P, sigma2, rho):
    return la.build_factor(P.locs, P.order, P.cov, sigma2, rho, P.m, 1e-10 * sigma2)


@pytest.mark.parametrize("lik", [la.LIK_BERNOULLI_LOGIT, la.LIK_POISSON_LOG])
def test_w_prime_is_the_derivative_of_w(lik):
    mu = np.linspace(-2.5, 2.0, 19)
    y = np.ones_like(mu)
    h = 1e-5
    d = (la.W_lik(y, mu + h, lik) - la.W_lik(y, mu - h, lik)) / (2 * h)
    assert np.allclose(gr.W_prime(y, mu, lik), d, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("cov", [vecchia.COV_EXPONENTIAL, vecchia.COV_MATERN15])
@pytest.mark.parametrize("par", gr.PARAMS)
def test_factor_derivatives_match_central_differences(cov, par):
    P = wl.tiny_problem(90, 7, cov=cov, rho=0.2)
    f = _factor(P, 1.3, 0.2)
    dA, dD = gr.factor_derivatives(f, par)
    # h balances truncation (O(h^2)) against rounding of the m x m solves (~1e-12 / h)
    h = 1e-4
    s2p, s2m = (1.3 + h, 1.3 - h) if par == "sigma2" else (1.3, 1.3)
    rp, rm = (0.2, 0.2) if par == "sigma2" else (0.2 + h, 0.2 - h)
    fp, fm = _factor(P, s2p, rp), _factor(P, s2m, rm)
    assert np.allclose(dA, (fp.A - fm.A) / (2 * h), rtol=1e-4, atol=1e-6)
    assert np.allclose(dD, (fp.D - fm.D) / (2 * h), rtol=1e-5, atol=1e-8)
    if par == "sigma2":      # A is invariant to sigma2 when the nugget follows it
        assert np.max(np.abs(dA)) < 1e-9


@pytest.mark.parametrize("lik,cov", [(la.LIK_BERNOULLI_LOGIT, vecchia.COV_EXPONENTIAL),
                                     (la.LIK_POISSON_LOG, vecchia.COV_MATERN15)])
def test_exact_gradient_matches_central_differences_of_the_laplace_value(lik, cov):
    """dL^VLA/dtheta including the implicit dependence through the mode."""
    P = wl.tiny_problem(120, 10, cov=cov, lik=lik, rho=0.15)
    s2, rho = 1.1, 0.15

    def L(s2_, rho_):
        f_ = _factor(P, s2_, rho_)
        md_ = la.find_mode(f_, P.y, P.F, lik, newton_tol=1e-14)
        return la.lml_exact(f_, md_)[0]

    f = _factor(P, s2, rho)
    md = la.find_mode(f, P.y, P.F, lik, newton_tol=1e-14)
    g = gr.lml_grad_exact(f, md)
    h = 1e-5
    fd = {"sigma2": (L(s2 + h, rho) - L(s2 - h, rho)) / (2 * h), "rho": (L(s2, rho + h) - L(s2, rho - h)) / (2 * h)}
    for par in gr.PARAMS:
        assert abs(g[par] - fd[par]) < 1e-5 * (1 + abs(fd[par])), (par, g[par], fd[par])


def test_ste_log_det_derivative_is_unbiased_and_the_control_variate_reduces_variance():
    P = wl.tiny_problem(100, 8, rho=0.2)
    f = _factor(P, P.sigma2, P.rho)
    md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-13)
    exact = gr.dlogdet_exact(f, md)
    t = 1500
    out = gr.lml_grad_ste(f, md, t, 3)
    plain = gr.lml_grad_ste(f, md, t, 3, control_variate=False)
    for par in gr.PARAMS:
        s = out["samples"][par]
        h, r, c = s["h"], s["r"], s["c"]
        se = np.std(h - c * r, ddof=1) / np.sqrt(t)
        assert abs(s["dlogdet"] - exact[par]) < 4 * se + 1e-12
        assert np.var(h - c * r) <= np.var(h) + 1e-15
        se0 = np.std(plain["samples"][par]["h"], ddof=1) / np.sqrt(t)
        assert abs(plain["samples"][par]["dlogdet"] - exact[par]) < 4 * se0 + 1e-12
    grad_ex = gr.lml_grad_exact(f, md)
    for par in gr.PARAMS:   # the full STE gradient, implicit term included, within its standard error
        pp = out["samples"][par]["per_probe"]
        assert abs(out["grad"][par] - grad_ex[par]) < 4 * np.std(pp, ddof=1) / np.sqrt(t) + 1e-12
    # sigma2's control variate is constant under Rademacher probes: its weight must be 0
    assert out["samples"]["sigma2"]["c"] == 0.0


def test_offset_gradient_matches_central_differences():
    """dL^VLA/dF_i (implicit mode term included) for a few coordinates."""
    P = wl.tiny_problem(110, 9, lik=la.LIK_POISSON_LOG, rho=0.2, F0=0.3)
    f = _factor(P, P.sigma2, P.rho)

    def L(F):
        md_ = la.find_mode(f, P.y, F, P.lik, newton_tol=1e-14)
        return la.lml_exact(f, md_)[0]

    md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-14)
    dF = gr.lml_grad_F_exact(f, md)
    h = 1e-5
    for i in (0, 17, 56, 109):
        e = np.zeros(P.n)
        e[i] = h
        fd = (L(P.F + e) - L(P.F - e)) / (2 * h)
        assert abs(dF[i] - fd) < 1e-6 * (1 + abs(fd)), (i, dF[i], fd)
    # the STE form with many probes tracks the exact one
    ste = gr.lml_grad_ste(f, md, 2000, 5)["grad"]["F"]
    assert np.max(np.abs(ste - dF)) < 0.05 * np.max(np.abs(dF))


# --------------------------------------------------------------------------- LRAC form
def test_lowrank_product_is_nystrom_and_its_derivative_matches_central_differences():
    """L_k L_k^T of the pivoted Cholesky equals Sigma_{:,I} Sigma_{I,I}^{-1} Sigma_{I,:} on its
    pivots, and d(L_k L_k^T)/dtheta at fixed pivots matches central differences of the
    pivoted Cholesky itself (whose pivots do not move under the perturbation)."""
    from oracle import lrac
    P = wl.tiny_problem(70, 8, rho=0.2)
    f = _factor(P, 1.2, 0.2)
    k = 12
    L, piv = lrac.pivoted_cholesky(f.locs, f.cov, f.sigma2, f.rho, f.nugget, k)
    S = vecchia.dense_cov(f.locs, f.cov, f.sigma2, f.rho, f.nugget)
    ny = S[:, piv] @ np.linalg.solve(S[np.ix_(piv, piv)], S[piv])
    assert np.max(np.abs(L @ L.T - ny)) < 1e-10 * np.max(np.abs(ny))
    h = 1e-5
    for par in gr.PARAMS:
        s2p, s2m = (1.2 + h, 1.2 - h) if par == "sigma2" else (1.2, 1.2)
        rp, rm = (0.2, 0.2) if par == "sigma2" else (0.2 + h, 0.2 - h)
        Lp, pp = lrac.pivoted_cholesky(f.locs, f.cov, s2p, rp, 1e-10 * s2p, k)
        Lm, pm = lrac.pivoted_cholesky(f.locs, f.cov, s2m, rm, 1e-10 * s2m, k)
        assert np.array_equal(pp, piv) and np.array_equal(pm, piv)
        fd = (Lp @ Lp.T - Lm @ Lm.T) / (2 * h)
        dLL = gr.lowrank_derivative(f, piv, par)
        assert np.max(np.abs(dLL - fd)) < 1e-6 * max(1.0, np.max(np.abs(fd))), par
    # sigma2 scales Sigma (the nugget follows it), so d(LL^T)/dsigma2 = LL^T / sigma2
    assert np.max(np.abs(gr.lowrank_derivative(f, piv, "sigma2") - L @ L.T / 1.2)) < 1e-12


def test_lrac_ste_gradient_is_unbiased_with_the_control_variate():
    P = wl.tiny_problem(90, 8, lik=la.LIK_POISSON_LOG, rho=0.2, F0=0.3)
    f = _factor(P, P.sigma2, P.rho)
    md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-13)
    t, k = 1500, 10
    out = gr.lml_grad_ste_lrac(f, md, k, t, 4)
    plain = gr.lml_grad_ste_lrac(f, md, k, t, 4, control_variate=False)
    exact = gr.dlogdet_exact(f, md)
    grad_ex = gr.lml_grad_exact(f, md)
    for par in gr.PARAMS:
        s = out["samples"][par]
        h, r, c = s["h"], s["r"], s["c"]
        # the control variate has the stated mean tr(P^{-1} d(LL^T))
        assert abs(r.mean() - s["tr_dlogP"]) < 4 * r.std(ddof=1) / np.sqrt(t) + 1e-12
        se = np.std(h - c * r, ddof=1) / np.sqrt(t)
        assert abs(s["dlogdet"] - exact[par]) < 4 * se + 1e-12, par
        assert np.var(h - c * r) <= np.var(h) + 1e-15
        s0 = plain["samples"][par]
        assert abs(s0["dlogdet"] - exact[par]) < 4 * np.std(s0["h"], ddof=1) / np.sqrt(t) + 1e-12
        pp = s["per_probe"]
        assert abs(out["grad"][par] - grad_ex[par]) < 4 * np.std(pp, ddof=1) / np.sqrt(t) + 1e-12, par
    # d logdet / d mu_j against (A^{-1})_jj W'_j, row by row within four standard errors
    Ainv = np.linalg.inv(np.diag(md.W) + f.Sinv.toarray())
    ex_mu = np.diag(Ainv) * gr.W_prime(md.y, md.mu, md.lik)
    sm = out["samples"]["mu"]
    dev = sm["h"] - sm["c"][:, None] * sm["r"]
    se_mu = dev.std(axis=1, ddof=1) / np.sqrt(t)
    assert np.all(np.abs(sm["dlogdet"] - ex_mu) < 4 * se_mu + 1e-12)
    # the offset gradient tracks the exact one
    dF = gr.lml_grad_F_exact(f, md)
    assert np.max(np.abs(out["grad"]["F"] - dF)) < 0.05 * np.max(np.abs(dF))
