"""Pins of the oracle's gamma likelihood (Section 5: y | mu ~ Gamma(alpha, alpha e^{-mu}),
E[y | mu] = e^mu), of the gradient in its shape parameter xi = alpha (appendix "Gradients
of Vecchia-Laplace approximations") and of the fixed-effect gradient dL/dbeta = X^T dL/dF
(Section 2). Each is checked against something other than the oracle's own formulas:
scipy's gamma density, numerical quadrature, central differences of scipy's density or
of the exact L^VLA, and the dense textbook Laplace approximation."""
import numpy as np
import pytest
from scipy import integrate, stats

import workloads as wl
from oracle import gradients as gr, laplace as la, textbook, vecchia

G = la.LIK_GAMMA_LOG


def _scipy_logpdf(y, mu, a):
    return stats.gamma.logpdf(y, a, scale=np.exp(mu) / a)


def _factor(P, sigma2=None, rho=None):
    s2 = P.sigma2 if sigma2 is None else sigma2
    return la.build_factor(P.locs, P.order, P.cov, s2, P.rho if rho is None else rho, P.m, 1e-10 * s2)


def test_gamma_log_density_is_scipys_and_has_mean_e_mu():
    rng = np.random.default_rng(0)
    y = rng.gamma(2.0, 1.0, 40) + 1e-3
    mu = rng.uniform(-2.0, 2.0, 40)
    for a in (0.7, 1.0, 6.5, 28.0):
        assert np.allclose(la.log_lik(y, mu, G, a), _scipy_logpdf(y, mu, a), rtol=1e-12, atol=1e-12)
    # normalisation and the mean fixed by the parametrisation, by quadrature
    for a, m0 in ((1.5, -0.7), (6.0, 0.4), (28.0, 1.2)):
        dens = lambda v: np.exp(la.log_lik(np.array([v]), np.array([m0]), G, a)[0])
        tot = integrate.quad(dens, 0.0, np.inf, limit=400)[0]
        mean = integrate.quad(lambda v: v * dens(v), 0.0, np.inf, limit=400)[0]
        assert abs(tot - 1.0) < 1e-9 and abs(mean - np.exp(m0)) < 1e-8 * np.exp(m0)


def test_gamma_mu_and_shape_derivatives_match_central_differences_of_scipy():
    rng = np.random.default_rng(1)
    y = rng.gamma(3.0, 0.5, 25) + 1e-2
    mu = rng.uniform(-1.5, 1.5, 25)
    h = 1e-5
    for a in (0.8, 4.0, 28.0):
        d1 = (_scipy_logpdf(y, mu + h, a) - _scipy_logpdf(y, mu - h, a)) / (2 * h)
        assert np.allclose(la.grad_lik(y, mu, G, a), d1, rtol=1e-7, atol=1e-7)
        d2 = (_scipy_logpdf(y, mu + h, a) - 2 * _scipy_logpdf(y, mu, a) + _scipy_logpdf(y, mu - h, a)) / h**2
        assert np.allclose(la.W_lik(y, mu, G, a), -d2, rtol=1e-4, atol=1e-4)
        d3 = (la.W_lik(y, mu + h, G, a) - la.W_lik(y, mu - h, G, a)) / (2 * h)
        assert np.allclose(gr.W_prime(y, mu, G, a), d3, rtol=1e-7, atol=1e-9)
        da = (_scipy_logpdf(y, mu, a + h) - _scipy_logpdf(y, mu, a - h)) / (2 * h)
        assert np.allclose(gr.dloglik_dxi(y, mu, G, a), da, rtol=1e-6, atol=1e-7)
        dam = (la.grad_lik(y, mu, G, a + h) - la.grad_lik(y, mu, G, a - h)) / (2 * h)
        assert np.allclose(gr.d2loglik_dxi_dmu(y, mu, G, a), dam, rtol=1e-7, atol=1e-8)
        dW = (la.W_lik(y, mu, G, a + h) - la.W_lik(y, mu, G, a - h)) / (2 * h)
        assert np.allclose(gr.dW_dxi(y, mu, G, a), dW, rtol=1e-7, atol=1e-9)
    with pytest.raises(ValueError):
        gr.dW_dxi(y, mu, la.LIK_POISSON_LOG, 1.0)


def test_gamma_full_conditioning_matches_textbook_laplace():
    P = wl.tiny_problem(70, 69, lik=G, rho=0.25, sigma2=0.4, seed=11, n_test=9, xi=6.0, beta=[0.5, 0.3, -0.2])
    f = _factor(P)
    md = la.find_mode(f, P.y, P.F, G, newton_tol=1e-12, xi=P.xi)
    L_ex, _ = la.lml_exact(f, md)
    K = vecchia.dense_cov(P.locs, P.cov, P.sigma2, P.rho, P.nugget)
    fb, nlml, Lc, W = textbook.gp_laplace(K, P.y, P.F, G, xi=P.xi)
    assert abs(L_ex - nlml) < 1e-10 * abs(nlml)
    assert np.max(np.abs(la.mode_user(f, md) - fb)) < 1e-9 * (1 + np.max(np.abs(fb)))
    pf = la.pred_factor(f, P.test_locs, 70)
    Ks = vecchia.cov_fn(vecchia.dist(P.locs[:, None, :], P.test_locs[None, :, :]), P.cov, P.sigma2, P.rho)
    mean_tb, var_tb = textbook.gp_predict(K, Ks, np.full(9, P.sigma2 + P.nugget), P.y, P.F, P.Fp, fb, Lc, W, G,
                                          xi=P.xi)
    assert np.allclose(la.pred_mean(pf, md, P.Fp), mean_tb, rtol=1e-8, atol=1e-9)
    assert np.allclose(la.pred_var_exact(f, md, pf), var_tb, rtol=1e-7, atol=1e-10)


def test_gamma_one_point_closed_form():
    """n = 1: the mode is the root of alpha (y e^{-(F+b)} - 1) - b / s2 and the Laplace value
    is -log p(y | F + b*) + b*^2 / (2 s2) + log(1 + s2 alpha y e^{-(F+b*)}) / 2."""
    from scipy.optimize import brentq
    s2, F, a = 0.8, 0.3, 5.0
    for yv in (0.05, 1.0, 7.5):
        root = lambda b: a * (yv * np.exp(-(F + b)) - 1.0) - b / s2
        b = brentq(root, -30.0, 30.0, xtol=1e-15, rtol=1e-15)
        ref = -float(_scipy_logpdf(yv, F + b, a)) + b * b / (2 * s2) + 0.5 * np.log1p(s2 * a * yv * np.exp(-(F + b)))
        f, nlml, _, _ = textbook.gp_laplace(np.array([[s2]]), np.array([yv]), np.array([F]), G, xi=a)
        assert abs(f[0] - b) < 1e-10 and abs(nlml - ref) < 1e-12 * (1 + abs(ref))


def _problem():
    return wl.tiny_problem(110, 9, lik=G, rho=0.18, sigma2=0.5, seed=5, xi=4.0, beta=[0.2, 0.6, -0.4])


def _L(P, s2, rho, xi, F):
    f = _factor(P, s2, rho)
    md = la.find_mode(f, P.y, F, G, newton_tol=1e-14, xi=xi)
    return la.lml_exact(f, md)[0]


def test_gamma_covariance_and_shape_gradients_match_central_differences():
    P = _problem()
    f = _factor(P)
    md = la.find_mode(f, P.y, P.F, G, newton_tol=1e-14, xi=P.xi)
    g = gr.lml_grad_exact(f, md)
    gx = gr.lml_grad_xi_exact(f, md)
    h = 1e-5
    fd = {"sigma2": (_L(P, P.sigma2 + h, P.rho, P.xi, P.F) - _L(P, P.sigma2 - h, P.rho, P.xi, P.F)) / (2 * h),
          "rho": (_L(P, P.sigma2, P.rho + h, P.xi, P.F) - _L(P, P.sigma2, P.rho - h, P.xi, P.F)) / (2 * h)}
    for par in gr.PARAMS:
        assert abs(g[par] - fd[par]) < 1e-5 * (1 + abs(fd[par])), (par, g[par], fd[par])
    fx = (_L(P, P.sigma2, P.rho, P.xi + h, P.F) - _L(P, P.sigma2, P.rho, P.xi - h, P.F)) / (2 * h)
    assert abs(gx - fx) < 1e-6 * (1 + abs(fx)), (gx, fx)
    # the implicit term matters: without it the derivative is off
    Ainv = np.linalg.inv(np.diag(md.W) + f.Sinv.toarray())
    g_mu = 0.5 * np.diag(Ainv) * gr.W_prime(md.y, md.mu, G, md.xi)
    implicit = float((Ainv @ g_mu) @ gr.d2loglik_dxi_dmu(md.y, md.mu, G, md.xi))
    assert abs(implicit) > 1e3 * 1e-6 * (1 + abs(fx))


def test_fixed_effect_gradient_is_x_transpose_offset_gradient():
    P = _problem()
    f = _factor(P)
    md = la.find_mode(f, P.y, P.F, G, newton_tol=1e-14, xi=P.xi)
    gb = gr.lml_grad_beta(P.X, gr.lml_grad_F_exact(f, md))
    h = 1e-5
    for k in range(len(P.beta)):
        e = np.zeros(len(P.beta))
        e[k] = h
        fd = (_L(P, P.sigma2, P.rho, P.xi, P.X @ (P.beta + e)) - _L(P, P.sigma2, P.rho, P.xi, P.X @ (P.beta - e))) / (2 * h)
        assert abs(gb[k] - fd) < 1e-6 * (1 + abs(fd)), (k, gb[k], fd)


def test_gamma_ste_shape_gradient_is_unbiased_with_the_control_variate():
    P = _problem()
    f = _factor(P)
    md = la.find_mode(f, P.y, P.F, G, newton_tol=1e-13, xi=P.xi)
    t = 1500
    out = gr.lml_grad_ste(f, md, t, 9)
    s = out["samples"]["xi"]
    Ainv = np.linalg.inv(np.diag(md.W) + f.Sinv.toarray())
    exact_dld = float(np.sum(np.diag(Ainv) * gr.dW_dxi(md.y, md.mu, G, md.xi)))
    se = np.std(s["h"] - s["c"] * s["r"], ddof=1) / np.sqrt(t)
    assert abs(s["dlogdet"] - exact_dld) < 4 * se + 1e-12
    assert np.var(s["h"] - s["c"] * s["r"]) <= np.var(s["h"]) + 1e-15
    se_g = np.std(s["per_probe"], ddof=1) / np.sqrt(t)
    assert abs(out["grad"]["xi"] - gr.lml_grad_xi_exact(f, md)) < 4 * se_g + 1e-12
    grad_ex = gr.lml_grad_exact(f, md)
    for par in gr.PARAMS:
        pp = out["samples"][par]["per_probe"]
        assert abs(out["grad"][par] - grad_ex[par]) < 4 * np.std(pp, ddof=1) / np.sqrt(t) + 1e-12
