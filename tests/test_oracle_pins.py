"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a library
routine implementing the same published definition, a closed form, a special
case that reduces to a textbook route, an invariant of a theorem in the paper,
or brute force on a tiny input.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.special as ss

import workloads as wl
from oracle import geometry, krylov, laplace as la, lrac, rng as orng, textbook, vecchia

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- rng
@pytest.mark.parametrize("ctr,key", [((0, 0, 0, 0), (0, 0)), ((5, 0, 0, 0), (7, 9)),
                                     ((2**64 - 2, 3, 2**63, 1), (2**64 - 1, 12345))])
def test_philox_matches_numpy_generator(ctr, key):
    # numpy's Philox bit generator implements Philox4x64-10 and increments the
    # counter before producing each 4-word block.
    bg = np.random.Philox(counter=np.array(ctr, np.uint64), key=np.array(key, np.uint64))
    ref = [int(v) for v in bg.random_raw(8)]
    c1 = list(ctr)
    out = []
    for _ in range(2):
        c1[0] += 1
        carry = 0
        for w in range(4):   # propagate the increment's carry
            c1[w] += carry
            carry = c1[w] >> 64
            c1[w] &= (1 << 64) - 1
        out += list(orng.philox4x64_10_scalar(c1, key))
        vec = orng.philox4x64_10(np.array([c1[0]], np.uint64), c1[1], c1[2], c1[3], key[0], key[1])
        assert [int(v[0]) for v in vec] == list(orng.philox4x64_10_scalar(c1, key))
    assert out == ref


def test_rademacher_and_gaussian_distribution():
    pts = np.arange(20000)
    r = orng.rademacher(pts, 300, seed=9)
    assert set(np.unique(r)) == {-1.0, 1.0}
    assert abs(r.mean()) < 4 / math.sqrt(r.size)
    # columns beyond 256 use the next counter block and are not copies of the first
    assert np.abs(r[:, 260] @ r[:, 4]) < 4 * math.sqrt(len(pts))
    z = orng.gaussian(pts, 7, seed=9, stream=orng.STREAM_SIM1)
    from scipy import stats
    for j in range(7):
        assert stats.kstest(z[:, j], "norm").pvalue > 1e-4
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 0.05
    z2 = orng.gaussian(pts, 7, seed=9, stream=orng.STREAM_SIM2)
    assert abs(np.corrcoef(z[:, 3], z2[:, 3])[0, 1]) < 0.05


# --------------------------------------------------------------------------- neighbours
def test_knn_golden_ties():
    g = json.load(open(os.path.join(GOLDEN, "knn_ties_m3.json")))
    locs = np.array(g["locs"])
    N = geometry.knn_prev(locs, g["m"])
    assert N.tolist() == g["N"]
    assert geometry.levels_forward(N).tolist() == g["lev_forward"]
    assert geometry.levels_backward(N).tolist() == g["lev_backward"]


def test_knn_prev_matches_kdtree_prefix_queries():
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(0)
    locs = rng.random((700, 2))
    m = 12
    N = geometry.knn_prev(locs, m)
    for i in [0, 1, 2, 5, 12, 13, 50, 400, 699]:
        k = min(i, m)
        if k == 0:
            assert (N[i] == -1).all()
            continue
        _, idx = cKDTree(locs[:i]).query(locs[i], k=k)
        assert sorted(np.atleast_1d(idx).tolist()) == sorted(N[i, :k].tolist())
        assert (N[i, k:] == -1).all()
        # ascending distance order inside the row
        d = np.hypot(*(locs[N[i, :k]] - locs[i]).T)
        assert np.all(np.diff(d) >= 0)


def test_knn_prev_fast_equals_brute_force_with_grid_ties():
    rng = np.random.default_rng(1)
    g = np.stack(np.meshgrid(np.arange(70), np.arange(70), indexing="ij"), -1).reshape(-1, 2) / 70.0
    locs = g[rng.permutation(len(g))]
    N_fast = la.knn_prev_fast(locs, 10)
    rows = np.concatenate([np.arange(40), rng.choice(len(g), 300, replace=False)])
    N_brute = geometry.knn_prev_rows(locs, 10, rows)
    assert np.array_equal(N_fast[rows], N_brute)


def test_knn_cross_matches_kdtree():
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(2)
    tr, te = rng.random((500, 2)), rng.random((60, 2))
    Np = geometry.knn_cross(tr, te, 9)
    _, idx = cKDTree(tr).query(te, k=9)
    assert np.array_equal(np.sort(Np, 1), np.sort(idx, 1))


def test_levels_equal_topological_generations():
    import networkx as nx
    rng = np.random.default_rng(3)
    locs = rng.random((300, 2))
    N = geometry.knn_prev(locs, 6)
    G = nx.DiGraph()
    G.add_nodes_from(range(len(N)))
    for i in range(len(N)):
        for j in N[i][N[i] >= 0]:
            G.add_edge(int(j), int(i))
    fwd = np.zeros(len(N), int)
    for gen, nodes in enumerate(nx.topological_generations(G)):
        fwd[list(nodes)] = gen
    bwd = np.zeros(len(N), int)
    for gen, nodes in enumerate(nx.topological_generations(G.reverse())):
        bwd[list(nodes)] = gen
    assert np.array_equal(geometry.levels_forward(N), fwd)
    assert np.array_equal(geometry.levels_backward(N), bwd)


# --------------------------------------------------------------------------- covariance / factor
@pytest.mark.parametrize("cov,nu", [(vecchia.COV_EXPONENTIAL, 0.5), (vecchia.COV_MATERN15, 1.5)])
def test_covariance_is_matern_bessel_form(cov, nu):
    # general Matern: sigma2 2^{1-nu}/Gamma(nu) (sqrt(2 nu) h/rho)^nu K_nu(sqrt(2 nu) h/rho)
    h = np.linspace(1e-3, 0.6, 50)
    rho, s2 = 0.11, 1.7
    a = math.sqrt(2 * nu) * h / rho
    ref = s2 * 2 ** (1 - nu) / ss.gamma(nu) * a ** nu * ss.kv(nu, a)
    assert np.allclose(vecchia.cov_fn(h, cov, s2, rho), ref, rtol=1e-12, atol=0)
    assert vecchia.cov_fn(np.array([0.0]), cov, s2, rho)[0] == s2


@pytest.mark.parametrize("cov", [vecchia.COV_EXPONENTIAL, vecchia.COV_MATERN15])
def test_factor_full_conditioning_is_exact_inverse(cov):
    P = wl.tiny_problem(150, 149, cov=cov, rho=0.3)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    S = vecchia.dense_cov(f.locs, cov, P.sigma2, P.rho, P.nugget)
    Sinv = np.linalg.inv(S)
    assert np.linalg.norm(f.Sinv.toarray() - Sinv) / np.linalg.norm(Sinv) < 1e-9
    # det B = 1, D > 0; log det Sigma = sum log D
    assert np.allclose(f.B.diagonal(), 1.0)
    assert (f.D > 0).all()
    assert abs(np.sum(np.log(f.D)) - np.linalg.slogdet(S)[1]) < 1e-9 * abs(np.linalg.slogdet(S)[1])


def test_factor_no_neighbours_is_diagonal():
    P = wl.tiny_problem(40, 0)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, 0, P.nugget)
    assert np.array_equal(f.B.toarray(), np.eye(40))
    assert np.allclose(f.D, P.sigma2 + P.nugget, rtol=0, atol=0)


def test_factor_rows_are_conditional_distributions():
    # For S = N(i) + {i}: the conditional of b_i given b_N(i) under N(0, Sigma_SS)
    # has precision Q_ii and mean -Q_iN / Q_ii b_N with Q = Sigma_SS^{-1}.
    P = wl.tiny_problem(120, 7, rho=0.15)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    for i in [1, 5, 7, 8, 60, 119]:
        nb = f.N[i][f.N[i] >= 0]
        S = np.concatenate([nb, [i]])
        Q = np.linalg.inv(vecchia.dense_cov(f.locs[S], P.cov, P.sigma2, P.rho, P.nugget))
        assert abs(f.D[i] - 1.0 / Q[-1, -1]) < 1e-10 * f.D[i]
        assert np.allclose(f.A[i, :len(nb)], -Q[-1, :-1] / Q[-1, -1], rtol=1e-8, atol=1e-10)


# --------------------------------------------------------------------------- Krylov
def _dense_M(f, W, prec):
    Bd = f.B.toarray()
    Bi = np.linalg.inv(Bd)
    A = np.diag(W) + f.Sinv.toarray()
    s = la.precond_scale(f, W, prec)
    return s[:, None] * (Bi.T @ A @ Bi) * s[None, :]


def test_pcg_T_equals_lanczos_T_and_spectrum():
    P = wl.tiny_problem(40, 4, rho=0.25)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik)
    A = np.diag(md.W) + f.Sinv.toarray()
    Pm = f.B.T.toarray() @ np.diag(md.W + 1 / f.D) @ f.B.toarray()
    r = orng.rademacher(f.order, 1, 4)[:, 0]
    s = la.precond_scale(f, md.W, la.PREC_VADU)
    z = f.B.T @ (r / s)                       # z = P^{1/2} r
    u, dT, oT, it, rel, r0z0 = krylov.pcg_with_T(lambda v: A @ v, lambda v: np.linalg.solve(Pm, v), z, 1e-13, 200)
    assert np.allclose(A @ u, z, rtol=0, atol=1e-10 * np.linalg.norm(z))
    assert abs(r0z0 - 40.0) < 1e-9               # ||P^{-1/2} z||^2 = ||r||^2 = n
    M = _dense_M(f, md.W, la.PREC_VADU)
    g, dL, oL = krylov.lanczos_fr(lambda v: M @ v, r.copy(), rtol=0.0, max_iter=len(dT))
    k = min(len(dT), len(dL), 8)
    assert np.allclose(dT[:k], dL[:k], rtol=1e-8)
    assert np.allclose(oT[:k - 1], oL[:k - 1], rtol=1e-7)
    # quadrature against a dense matrix logarithm
    assert abs(krylov.quad_log(dT, oT, 40.0) - 40.0 * sla.logm(krylov.tridiag(dT, oT))[0, 0].real) < 1e-9
    # at full length the Ritz values are the spectrum of the preconditioned matrix
    ev_T = np.linalg.eigvalsh(krylov.tridiag(dL, oL)) if len(dL) == 40 else None
    if ev_T is not None:
        assert np.allclose(np.sort(ev_T), np.linalg.eigvalsh(M), rtol=1e-8)


def test_vadu_identity_factor_gives_exact_one_step():
    # B = I (m = 0): the VADU-preconditioned matrix is I (Section 3.1.1)
    P = wl.tiny_problem(50, 0)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, 0, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik)
    M = _dense_M(f, md.W, la.PREC_VADU)
    assert np.allclose(M, np.eye(50), atol=1e-13)
    _, ld, g = la.lml_slq(f, md, 6, 2)
    assert np.allclose(g, 0.0, atol=1e-12)
    assert abs(ld - np.sum(np.log1p(f.D * md.W))) < 1e-11
    A = np.diag(md.W) + f.Sinv.toarray()
    Pm = np.diag(md.W + 1 / f.D)
    *_, it, rel, _ = krylov.pcg_with_T(lambda v: A @ v, lambda v: np.linalg.solve(Pm, v), np.ones(50), 1e-12, 10)
    assert it == 1


def test_lva_identity_factor_closed_form():
    """m = 0: B = I and D = diag(Sigma), so P_LVA = D^{-1} and the preconditioned matrix is
    D^{1/2} (W + D^{-1}) D^{1/2} = I + D W (Section 3.1.1). Every Rademacher probe then gives
    gamma_i = sum_j r_j^2 log(1 + D_j W_j) = sum_j log(1 + D_j W_j) exactly, and the LVA split
    sum log D + log det P_LVA + gamma = sum log(1 + D W) is the exact log det(Sigma_tilde W + I).
    A sign error in log det P_LVA = -sum log D would move the total by 2 sum log D."""
    P = wl.tiny_problem(60, 0, lik=la.LIK_POISSON_LOG, rho=0.2, F0=0.4)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, 0, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-12)
    closed = float(np.sum(np.log1p(f.D * md.W)))
    L, ld, g = la.lml_slq(f, md, 7, 3, prec=la.PREC_LVA)
    assert np.allclose(g, closed, rtol=1e-12, atol=1e-12)
    assert abs(ld - closed) < 1e-12 * abs(closed)
    assert abs(la.logdet_P(f, md.W, la.PREC_LVA) + np.sum(np.log(f.D))) < 1e-12
    L_ex, ld_ex = la.lml_exact(f, md)
    assert abs(ld - ld_ex) < 1e-11 * abs(ld_ex) and abs(L - L_ex) < 1e-11 * abs(L_ex)


def test_lva_estimate_brackets_the_exact_logdet():
    """With neighbours (m = 6), the LVA split with a dense-eigendecomposition SLQ over 4000
    Rademacher probes lies within 4 standard errors of the exact log det(Sigma_tilde W + I), and
    the oracle's Lanczos gammas equal the dense quadratic forms r^T log(M_LVA) r."""
    P = wl.tiny_problem(120, 6, rho=0.25, seed=5)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-12)
    M = _dense_M(f, md.W, la.PREC_LVA)
    th, V = np.linalg.eigh(M)
    logM = (V * np.log(th)) @ V.T
    R = la.probes(f, 4000, seed=9)
    g_dense = np.einsum("ij,ij->j", R, logM @ R)
    base = float(np.sum(np.log(f.D))) + la.logdet_P(f, md.W, la.PREC_LVA)
    _, ld_ex = la.lml_exact(f, md)
    se = g_dense.std(ddof=1) / math.sqrt(len(g_dense))
    assert abs(base + g_dense.mean() - ld_ex) < 4 * se
    _, ld_slq, g = la.lml_slq(f, md, 6, 9, prec=la.PREC_LVA)
    assert np.allclose(g, g_dense[:6], rtol=1e-10, atol=1e-10)
    assert abs(ld_slq - (base + g.mean())) < 1e-10 * abs(ld_slq)


@pytest.mark.parametrize("prec", [la.PREC_VADU, la.PREC_LVA])
def test_theorem_3_1_eigenvalue_bounds(prec):
    P = wl.tiny_problem(200, 10, rho=0.2)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik)
    ev = np.linalg.eigvalsh(_dense_M(f, md.W, prec))
    St = np.linalg.inv(f.Sinv.toarray())
    lam_S = np.sort(np.linalg.eigvalsh(St))[::-1]
    if prec == la.PREC_VADU:
        assert ev.min() > np.min(1 / (f.D * md.W + 1)) * (1 - 1e-12)
        assert ev.max() <= (lam_S[0] * md.W.max() + 1) * np.max(1 / (f.D * md.W + 1)) * (1 + 1e-10)
    else:
        assert ev.min() > 1 - 1e-12
        assert ev.max() <= (lam_S[0] * md.W.max() + 1) * (1 + 1e-10)


def test_slq_gamma_equals_dense_quadratic_form_and_is_unbiased():
    P = wl.tiny_problem(100, 5, rho=0.3)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik)
    M = _dense_M(f, md.W, la.PREC_VADU)
    th, V = np.linalg.eigh(M)
    logM = (V * np.log(th)) @ V.T
    R = la.probes(f, 4000, seed=21)
    g_lanczos = la.slq_gammas(f, md, R[:, :5])
    g_dense = np.einsum("ij,ij->j", R, logM @ R)
    assert np.allclose(g_lanczos, g_dense[:5], rtol=1e-10, atol=1e-10)
    exact = np.sum(np.log(th))
    se = g_dense.std(ddof=1) / math.sqrt(len(g_dense))
    assert abs(g_dense.mean() - exact) < 4 * se
    # the full estimate brackets the exact log det(Sigma_tilde W + I)
    _, ld_ex = la.lml_exact(f, md)
    _, ld_slq, _ = la.lml_slq(f, md, 5, 21)
    assert abs(ld_slq - (np.sum(np.log(f.D)) + np.sum(np.log(md.W + 1 / f.D)) + g_lanczos.mean())) < 1e-9
    assert abs(np.sum(np.log(f.D)) + np.sum(np.log(md.W + 1 / f.D)) + exact - ld_ex) < 1e-8


# --------------------------------------------------------------------------- Laplace
@pytest.mark.parametrize("lik,cov", [(la.LIK_BERNOULLI_LOGIT, vecchia.COV_EXPONENTIAL),
                                     (la.LIK_POISSON_LOG, vecchia.COV_MATERN15)])
def test_full_conditioning_matches_textbook_laplace(lik, cov):
    P = wl.tiny_problem(80, 79, cov=cov, lik=lik, rho=0.25, seed=8, n_test=11, F0=0.3)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-12)
    L_ex, _ = la.lml_exact(f, md)
    K = vecchia.dense_cov(P.locs, cov, P.sigma2, P.rho, P.nugget)
    fb, nlml, Lc, W = textbook.gp_laplace(K, P.y, P.F, lik)
    assert abs(L_ex - nlml) < 1e-10 * abs(nlml)
    assert np.max(np.abs(la.mode_user(f, md) - fb)) < 1e-9 * (1 + np.max(np.abs(fb)))
    # prediction with every training point as neighbour
    pf = la.pred_factor(f, P.test_locs, 80)
    Ks = vecchia.cov_fn(vecchia.dist(P.locs[:, None, :], P.test_locs[None, :, :]), cov, P.sigma2, P.rho)
    mean_tb, var_tb = textbook.gp_predict(K, Ks, np.full(11, P.sigma2 + P.nugget), P.y, P.F, P.Fp, fb, Lc, W, lik)
    assert np.allclose(la.pred_mean(pf, md, P.Fp), mean_tb, rtol=1e-8, atol=1e-9)
    assert np.allclose(la.pred_var_exact(f, md, pf), var_tb, rtol=1e-7, atol=1e-10)


def test_mode_satisfies_stationarity_at_medium_n():
    P = wl.make_problem("c1_n2000")
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik)
    g = la.grad_lik(md.y, md.mu, md.lik) - f.Sinv @ md.b
    assert np.max(np.abs(g)) < 1e-9 * (1 + np.max(np.abs(la.grad_lik(md.y, md.mu, md.lik))))


def test_exact_logdet_matches_dense_and_no_neighbour_closed_form():
    P = wl.tiny_problem(300, 8, lik=la.LIK_POISSON_LOG, rho=0.1)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik)
    _, ld = la.lml_exact(f, md)
    St = np.linalg.inv(f.Sinv.toarray())
    assert abs(ld - np.linalg.slogdet(St * md.W[None, :] + np.eye(300))[1]) < 1e-9 * abs(ld)
    f0 = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, 0, P.nugget)
    md0 = la.find_mode(f0, P.y, P.F, P.lik)
    _, ld0 = la.lml_exact(f0, md0)
    assert abs(ld0 - np.sum(np.log1p(f0.D * md0.W))) < 1e-10 * abs(ld0)


def test_simulated_variances_are_unbiased():
    # Proposition 3.3: Algorithm simAlgo is unbiased; with many vectors it approaches
    # the exact diagonal within the central-limit bound.
    P = wl.tiny_problem(150, 6, rho=0.2, n_test=20)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik)
    pf = la.pred_factor(f, P.test_locs, 6)
    ex = la.pred_var_exact(f, md, pf)
    s = 4000
    sim = la.pred_var_sim(f, md, pf, s, seed=5)
    post = ex - pf.Dp                              # variance of z4 = Gaussian, var of z4^2 = 2 post^2
    assert np.all(np.abs(sim - ex) < 5 * np.sqrt(2.0) * post / math.sqrt(s) + 1e-12)
    assert np.all(sim >= pf.Dp)


# --------------------------------------------------------------------------- LRAC
def test_pivoted_cholesky_full_rank_reproduces_sigma():
    P = wl.tiny_problem(60, 5)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    L, piv = lrac.pivoted_cholesky(f.locs, P.cov, P.sigma2, P.rho, P.nugget, 60)
    S = vecchia.dense_cov(f.locs, P.cov, P.sigma2, P.rho, P.nugget)
    assert np.allclose(L @ L.T, S, atol=1e-10)
    assert sorted(piv.tolist()) == list(range(60)) and piv[0] == 0
    # the pivot rule makes L[piv] lower triangular: a permuted Cholesky factor
    assert np.allclose(np.triu(L[piv], 1), 0.0, atol=1e-14)


def test_lrac_woodbury_and_exact_limit():
    P = wl.tiny_problem(70, 69, rho=0.3)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik)
    L, _ = lrac.pivoted_cholesky(f.locs, P.cov, P.sigma2, P.rho, P.nugget, 25)
    Pm = L @ L.T + np.diag(1 / md.W)
    X = np.random.default_rng(0).standard_normal((70, 3))
    assert np.allclose(lrac.woodbury_apply(L, md.W, X), np.linalg.solve(Pm, X), rtol=1e-9, atol=1e-9)
    assert abs(lrac.logdet_P(L, md.W) - np.linalg.slogdet(Pm)[1]) < 1e-9
    # m = n - 1 and k = n: P = Sigma_tilde + W^{-1}, so SLQ_2 = 0 and the estimate is exact
    Lf, ldf, g = lrac.lml_lrac_dense(f, md, 70, 5, 3)
    assert np.allclose(g, 0.0, atol=1e-8)
    assert abs(Lf - la.lml_exact(f, md)[0]) < 1e-8


def test_lrac_probes_have_covariance_P_and_slq_is_unbiased():
    """z = L r1 + W^{-1/2} r2 has E z z^T = P (Sec. 3.1.2 with Rademacher r1, r2), and the
    form-2 estimate log det C + mean gamma matches the exact log det(Sigma_tilde W + I)
    within four standard errors."""
    P = wl.tiny_problem(80, 10, rho=0.25)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik)
    k = 12
    L, _ = lrac.pivoted_cholesky(f.locs, P.cov, P.sigma2, P.rho, P.nugget, k)
    N = 4000
    Z = lrac.lrac_probes(f, L, md.W, N, 5)
    Pm = L @ L.T + np.diag(1.0 / md.W)
    # sampling error of the empirical covariance: E||C_N - P||_F^2 <= (tr(P)^2 + ||P||_F^2) / N
    # (the Gaussian value; Rademacher fourth moments are smaller). A wrong probe covariance
    # leaves an error that does not shrink with N.
    bound = np.sqrt((np.trace(Pm) ** 2 + np.linalg.norm(Pm) ** 2) / N)
    assert np.linalg.norm(Z @ Z.T / N - Pm) < 1.5 * bound
    _, ld, g = lrac.lml_lrac_dense(f, md, k, 400, 7)
    _, ld_ex = la.lml_exact(f, md)
    assert abs(ld - ld_ex) < 4 * g.std(ddof=1) / np.sqrt(len(g)) + 1e-9


# --------------------------------------------------------------------------- likelihood pieces
@pytest.mark.parametrize("lik", [la.LIK_BERNOULLI_LOGIT, la.LIK_POISSON_LOG])
def test_likelihood_derivatives_and_normalisation(lik):
    """grad and W are the first and negated second derivatives of log p (by central
    differences), and p(. | mu) sums to one over y, which pins the constant terms
    (-log y! for Poisson) that L^VLA includes."""
    mu = np.linspace(-3.0, 2.5, 23)
    y = (np.arange(23) % 2).astype(float) if lik == la.LIK_BERNOULLI_LOGIT else (np.arange(23) % 5).astype(float)
    h = 1e-5
    d1 = (la.log_lik(y, mu + h, lik) - la.log_lik(y, mu - h, lik)) / (2 * h)
    assert np.allclose(la.grad_lik(y, mu, lik), d1, rtol=1e-7, atol=1e-8)
    d2 = (la.grad_lik(y, mu + h, lik) - la.grad_lik(y, mu - h, lik)) / (2 * h)
    assert np.allclose(la.W_lik(y, mu, lik), -d2, rtol=1e-6, atol=1e-8)
    ys = np.arange(2.0) if lik == la.LIK_BERNOULLI_LOGIT else np.arange(400.0)
    for m0 in (-2.0, 0.3, 2.5):
        total = np.exp(la.log_lik(ys, np.full(len(ys), m0), lik)).sum()
        assert abs(total - 1.0) < 1e-12


@pytest.mark.parametrize("lik", [la.LIK_BERNOULLI_LOGIT, la.LIK_POISSON_LOG])
def test_textbook_laplace_one_point_closed_form(lik):
    """n = 1: the mode solves d/db [log p(y | F + b) - b^2 / (2 s2)] = 0 (a scalar root),
    and the Laplace value is -log p(y | F + b*) + b*^2 / (2 s2) + log(1 + s2 W(b*)) / 2."""
    from scipy.optimize import brentq
    s2, F = 1.7, 0.4
    for yv in ((0.0, 1.0) if lik == la.LIK_BERNOULLI_LOGIT else (0.0, 3.0, 11.0)):
        y = np.array([yv])
        g = lambda b: float(la.grad_lik(y, np.array([F + b]), lik)[0]) - b / s2
        b = brentq(g, -30.0, 30.0, xtol=1e-15, rtol=1e-15)
        W = float(la.W_lik(y, np.array([F + b]), lik)[0])
        ref = -float(la.log_lik(y, np.array([F + b]), lik)[0]) + b * b / (2 * s2) + 0.5 * np.log1p(s2 * W)
        f, nlml, _, _ = textbook.gp_laplace(np.array([[s2]]), y, np.array([F]), lik)
        assert abs(f[0] - b) < 1e-10 and abs(nlml - ref) < 1e-12 * (1 + abs(ref))


def test_refit_equals_a_fresh_factor():
    P = wl.tiny_problem(120, 8)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    g = la.refit(f, 2.5, 0.07, 3e-9)
    h = la.build_factor(P.locs, P.order, P.cov, 2.5, 0.07, P.m, 3e-9)
    assert np.array_equal(g.N, h.N) and np.allclose(g.A, h.A, rtol=0, atol=0) and np.allclose(g.D, h.D, rtol=0, atol=0)
    assert (g.sigma2, g.rho, g.nugget) == (2.5, 0.07, 3e-9)


@pytest.mark.parametrize("precond", [1, 2])
def test_lanczos_variances_are_exact_at_full_rank_and_converge(precond):
    """At k = n the preconditioned Lanczos factorisation is exact, so the variances equal
    the direct ones; with growing k the error falls."""
    from oracle import lanczos_pred as lp
    P = wl.tiny_problem(90, 10, rho=0.2, n_test=12)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik)
    pf = la.pred_factor(f, P.test_locs, P.m)
    exact = la.pred_var_exact(f, md, pf)
    full = lp.pred_var_lanczos(f, md, pf, 90, precond)
    assert np.allclose(full, exact, rtol=1e-8, atol=1e-10)
    errs = [np.max(np.abs(lp.pred_var_lanczos(f, md, pf, k, precond) - exact)) for k in (5, 20, 60)]
    assert errs[2] <= errs[1] <= errs[0] + 1e-12


@pytest.mark.parametrize("k", [3, 8, 15])
def test_lanczos_basis_invariants_and_cg_equivalence(k):
    """At any k the Lanczos basis is orthonormal, Q^T M Q = T, and ||v0|| Q T^{-1} e1 is the
    k-th CG iterate for M x = v0 from x = 0 (computed by the separate CG routine)."""
    from oracle import lanczos_pred as lp
    P = wl.tiny_problem(80, 8, lik=la.LIK_POISSON_LOG, rho=0.2)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik)
    lo, up = la._tri_solvers(f.B)
    s = la.precond_scale(f, md.W, la.PREC_VADU)
    Aap = la.A_apply_fn(f, md.W)
    M = lambda v: s * up(Aap(lo(s * v)))
    v0 = np.random.default_rng(2).standard_normal(P.n)
    Q, T = lp.lanczos_basis(M, v0, k)
    assert Q.shape == (P.n, k)
    assert np.max(np.abs(Q.T @ Q - np.eye(k))) < 1e-12
    MQ = np.column_stack([M(Q[:, j]) for j in range(k)])
    assert np.max(np.abs(Q.T @ MQ - T)) < 1e-10 * np.max(np.abs(T))
    x_l = np.linalg.norm(v0) * Q @ np.linalg.solve(T, np.eye(k)[:, 0])
    x_cg = krylov.pcg_with_T(M, lambda r: r, v0, 0.0, k)[0]
    assert np.linalg.norm(x_l - x_cg) < 1e-8 * np.linalg.norm(x_cg)
