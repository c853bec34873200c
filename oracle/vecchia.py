"""Covariance functions and the Vecchia factor, by definition (Section 2.1).

For each row i with neighbour set N(i):
    A_i = Sigma_{i,N(i)} Sigma_{N(i)}^{-1}
    D_i = Sigma_{i,i} - Sigma_{N(i),i}^T Sigma_{N(i)}^{-1} Sigma_{N(i),i}
B is unit lower triangular with B_{i,N(i)} = -A_i, D = diag(D_i), and
Sigma_tilde^{-1} = B^T D^{-1} B.

Covariances (Section 4.1 and the exponential member of the same family):
    Matern nu = 3/2:  c(h) = sigma2 (1 + sqrt(3) h / rho) exp(-sqrt(3) h / rho)
    exponential:      c(h) = sigma2 exp(-h / rho)
A nugget tau is added to every diagonal entry Sigma_{i,i} (the paper has none;
the default tau = 1e-10 sigma2 is a reading shared with the CUDA side).

Sigma_{N(i)} is solved with a dense LU solve (numpy.linalg.solve), one row at a
time in the paper's notation, batched over rows with equal |N(i)|.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

COV_EXPONENTIAL = 0
COV_MATERN15 = 1


def cov_fn(h: np.ndarray, cov: int, sigma2: float, rho: float) -> np.ndarray:
    if cov == COV_EXPONENTIAL:
        return sigma2 * np.exp(-h / rho)
    if cov == COV_MATERN15:
        a = math.sqrt(3.0) * h / rho
        return sigma2 * (1.0 + a) * np.exp(-a)
    raise ValueError(cov)


def dist(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Euclidean distances between the rows of a (..., 2) and b (..., 2)."""
    d = a - b
    return np.sqrt(d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1])


def vecchia_factor(locs: np.ndarray, N: np.ndarray, cov: int, sigma2: float, rho: float,
                   nugget: float):
    """Returns (A, D): A[i, :k_i] = A_i (aligned with N[i]), D[i] = D_i."""
    n, m = N.shape
    A = np.zeros((n, m))
    D = np.empty(n)
    k_of = (N >= 0).sum(1)
    for k in range(m + 1):
        rows = np.nonzero(k_of == k)[0]
        for a in range(0, len(rows), 8192):
            r = rows[a:a + 8192]
            sii = sigma2 + nugget
            if k == 0:
                D[r] = sii
                continue
            nb = N[r, :k]                                         # (R, k)
            P = locs[nb]                                          # (R, k, 2)
            S_NN = cov_fn(dist(P[:, :, None, :], P[:, None, :, :]), cov, sigma2, rho)
            S_NN[:, np.arange(k), np.arange(k)] += nugget
            S_Ni = cov_fn(dist(P, locs[r][:, None, :]), cov, sigma2, rho)   # (R, k)
            Ai = np.linalg.solve(S_NN, S_Ni[..., None])[..., 0]
            A[r, :k] = Ai
            D[r] = sii - (S_Ni * Ai).sum(1)
    return A, D


def B_matrix(N: np.ndarray, A: np.ndarray) -> sp.csr_matrix:
    n, m = N.shape
    rows = np.repeat(np.arange(n), m)
    cols = N.ravel()
    vals = -A.ravel()
    ok = cols >= 0
    off = sp.csr_matrix((vals[ok], (rows[ok], cols[ok])), shape=(n, n))
    return (sp.identity(n, format="csr") + off).tocsr()


def precision(B: sp.csr_matrix, D: np.ndarray) -> sp.csr_matrix:
    """Sigma_tilde^{-1} = B^T D^{-1} B."""
    return (B.T @ sp.diags(1.0 / D) @ B).tocsr()


def dense_cov(locs: np.ndarray, cov: int, sigma2: float, rho: float, nugget: float) -> np.ndarray:
    S = cov_fn(dist(locs[:, None, :], locs[None, :, :]), cov, sigma2, rho)
    S[np.diag_indices_from(S)] += nugget
    return S
