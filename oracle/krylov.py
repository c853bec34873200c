"""Krylov pieces of the method, written from the paper.

pcg_with_T   Preconditioned CG that also returns the Lanczos tridiagonal
             (Appendix, "Preconditioned conjugate gradient algorithm with Lanczos
             tridiagonal matrix"). Reading of its indexing: alpha_0 = 1,
             beta_0 = 0; after iteration l (0-based) the diagonal entry l is
             1/alpha_{l+1} + beta_l/alpha_l and, for l > 0, the off-diagonal
             entry (l-1, l) is sqrt(beta_l)/alpha_l; the stopping test on
             ||r_{l+1}|| comes before the T update, so T holds the last alpha.
             The test is relative: ||r_{l+1}|| <= tol * ||b||.
lanczos_fr   Explicit Lanczos with full reorthogonalisation of a symmetric
             operator from a start vector, run until the quadrature value
             ||v||^2 e1^T log(T) e1 stops changing (Section 3, Eq. def_SLQ and its
             derivation in the appendix).
quad_log     ||v||^2 e1^T log(T) e1 from a dense symmetric eigendecomposition of T.
"""
from __future__ import annotations

import numpy as np


def tridiag(diag, off) -> np.ndarray:
    l = len(diag)
    T = np.diag(np.asarray(diag, float))
    if l > 1:
        T += np.diag(np.asarray(off, float), 1) + np.diag(np.asarray(off, float), -1)
    return T


def quad_log(diag, off, norm2: float) -> float:
    """norm2 * e1^T log(T) e1 = norm2 * sum_j q_{1j}^2 log(theta_j)."""
    theta, Q = np.linalg.eigh(tridiag(diag, off))
    return float(norm2 * np.sum(Q[0, :] ** 2 * np.log(theta)))


def pcg_with_T(A_apply, Pinv_apply, b: np.ndarray, tol: float, max_iter: int):
    """Returns (u, diag_T, offdiag_T, n_iter, rel_res, r0z0)."""
    u = np.zeros_like(b)
    r = b - A_apply(u)
    z = Pinv_apply(r)
    h = z.copy()
    bnorm = np.linalg.norm(b)
    rz = float(r @ z)
    r0z0 = rz
    alpha_prev, beta_prev = 1.0, 0.0
    dT, oT = [], []
    rel = np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0
    if bnorm == 0.0:
        return u, np.zeros(0), np.zeros(0), 0, 0.0, 0.0
    it = 0
    for l in range(max_iter):
        v = A_apply(h)
        alpha = rz / float(h @ v)
        u = u + alpha * h
        r = r - alpha * v
        rel = np.linalg.norm(r) / bnorm
        stop = rel <= tol
        z = Pinv_apply(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        h = z + beta * h
        dT.append(1.0 / alpha + beta_prev / alpha_prev)
        if l > 0:
            oT.append(np.sqrt(beta_prev) / alpha_prev)
        alpha_prev, beta_prev, rz = alpha, beta, rz_new
        it = l + 1
        if stop:
            break
    return u, np.array(dT), np.array(oT), it, rel, r0z0


def lanczos_fr(M_apply, v0: np.ndarray, rtol: float = 1e-14, max_iter: int | None = None):
    """Lanczos with full reorthogonalisation. Returns (gamma, diag_T, offdiag_T)
    where gamma = ||v0||^2 e1^T log(T) e1 at convergence."""
    n = len(v0)
    max_iter = n if max_iter is None else min(max_iter, n)
    nrm2 = float(v0 @ v0)
    if nrm2 == 0.0:
        return 0.0, np.zeros(0), np.zeros(0)
    Q = np.zeros((n, max_iter))
    Q[:, 0] = v0 / np.sqrt(nrm2)
    alphas, betas = [], []
    gamma_prev = None
    gamma = 0.0
    scale = None
    for j in range(max_iter):
        w = M_apply(Q[:, j])
        a = float(Q[:, j] @ w)
        alphas.append(a)
        for _ in range(2):   # full reorthogonalisation, twice
            w = w - Q[:, :j + 1] @ (Q[:, :j + 1].T @ w)
        b = float(np.linalg.norm(w))
        gamma = quad_log(alphas, betas, nrm2)
        if scale is None:
            scale = max(abs(a), 1e-300)
        if gamma_prev is not None and abs(gamma - gamma_prev) <= rtol * (abs(gamma) + 1e-3 * nrm2):
            break
        if b <= 1e-13 * scale or j + 1 == max_iter:   # invariant subspace: exact
            break
        betas.append(b)
        Q[:, j + 1] = w / b
        gamma_prev = gamma
    return gamma, np.array(alphas), np.array(betas[: len(alphas) - 1])
