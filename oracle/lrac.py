"""LRAC preconditioner and the form-2 quantities (Section 3.1.2, Eqs. P_LRAC,
pcls2, logdetsplit2).

P_LRAC = L_k L_k^T + W^{-1}, L_k the rank-k pivoted Cholesky factor of the
original covariance Sigma (with the nugget on its diagonal), not Sigma_tilde.
Pivoted Cholesky (Harbrecht, Peters & Schneider 2012): keep the residual
diagonal d (initially diag Sigma); at step j take the pivot p = argmax d (ties to
the lowest Vecchia row index), set
    L[:, j] = (Sigma[:, p] - L[:, :j] L[p, :j]^T) / sqrt(d_p),  d <- d - L[:, j]^2,
and d_p <- 0; stop after exactly k steps.

Woodbury / determinant lemma:
    P^{-1} x = W x - W L (I_k + L^T W L)^{-1} L^T W x
    log det P = log det(I_k + L^T W L) - sum log W_i
Form 2 (Eq. logdetsplit2):
    log det(Sigma_tilde W + I) = log det W + log det P + log det(P^{-1/2} (W^{-1} + Sigma_tilde) P^{-T/2})
                               = log det(I_k + L^T W L) + SLQ_2.
Probes z = L r1 + W^{-1/2} r2 (r1 in {+-1}^k, r2 in {+-1}^n), so E[z z^T] = P; the SLQ
weight is ||P^{-1/2} z||^2 = z^T P^{-1} z.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import krylov, laplace, rng as orng, vecchia


def pivoted_cholesky(locs, cov, sigma2, rho, nugget, k):
    n = len(locs)
    k = min(k, n)
    d = np.full(n, sigma2 + nugget)
    L = np.zeros((n, k))
    piv = np.zeros(k, np.int64)
    for j in range(k):
        p = int(np.argmax(d))
        piv[j] = p
        if d[p] <= 0.0:
            raise FloatingPointError(f"pivoted Cholesky breakdown at step {j}")
        col = vecchia.cov_fn(vecchia.dist(locs, locs[p][None, :]), cov, sigma2, rho)
        col[p] += nugget
        col = col - L[:, :j] @ L[p, :j]
        L[:, j] = col / np.sqrt(d[p])
        d = d - L[:, j] ** 2
        d[p] = 0.0
    return L, piv


def woodbury_apply(L, W, X):
    WX = W[:, None] * X if X.ndim == 2 else W * X
    C = np.eye(L.shape[1]) + L.T @ (W[:, None] * L)
    return WX - (W[:, None] * L if X.ndim == 2 else W[:, None] * L) @ np.linalg.solve(C, L.T @ WX)


def logdet_P(L, W):
    C = np.eye(L.shape[1]) + L.T @ (W[:, None] * L)
    return float(np.linalg.slogdet(C)[1] - np.sum(np.log(W)))


def sigma_tilde_dense(f: laplace.Factor) -> np.ndarray:
    Binv = np.linalg.inv(f.B.toarray())
    return Binv @ np.diag(f.D) @ Binv.T


def lrac_probes(f: laplace.Factor, L, W, t, seed):
    r1 = orng.rademacher(np.arange(L.shape[1]), t, seed, orng.STREAM_PROBE_K)
    r2 = orng.rademacher(f.order, t, seed, orng.STREAM_PROBE)
    return L @ r1 + r2 / np.sqrt(W)[:, None]


def lml_lrac_dense(f: laplace.Factor, md: laplace.Mode, k: int, t: int, seed: int):
    """(L^VLA, logdet, gammas) with the form-2 same-probe SLQ and the LRAC
    preconditioner; dense linear algebra, so small n only."""
    L, _ = pivoted_cholesky(f.locs, f.cov, f.sigma2, f.rho, f.nugget, k)
    W = md.W
    St = sigma_tilde_dense(f)
    A2 = St + np.diag(1.0 / W)
    P = L @ L.T + np.diag(1.0 / W)
    C = np.linalg.cholesky(P)
    M = sla.solve_triangular(C, sla.solve_triangular(C, A2, lower=True).T, lower=True).T
    Z = lrac_probes(f, L, W, t, seed)
    g = []
    for j in range(t):
        v0 = sla.solve_triangular(C, Z[:, j], lower=True)
        g.append(krylov.lanczos_fr(lambda v: M @ v, v0)[0])
    g = np.array(g)
    Cl = np.eye(L.shape[1]) + L.T @ (W[:, None] * L)
    ld = float(np.linalg.slogdet(Cl)[1] + np.mean(g))
    p = laplace.lml_parts(f, md)
    return p["neg_loglik"] + p["quad"] + 0.5 * ld, ld, g
