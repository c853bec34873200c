"""Predictive variances by a preconditioned partial Lanczos factorisation (Section 4,
"Predictive (co-)variances using preconditioned Lanczos algorithms"). Test
infrastructure: a plain float64 CPU restatement; nothing here is used by the CUDA path.

With A = W + Sigma_tilde^{-1} and a preconditioner P = P^{1/2} P^{T/2}, k steps of the
Lanczos algorithm with full reorthogonalisation on M = P^{-1/2} A P^{-T/2} give
M ~ Q T Q^T (Q: n x k orthonormal, T: k x k tridiagonal), started from
P^{-1/2} times the mean of the columns of B_po^T B_p^{-1} (B_p = I here, Section 4.1
ordering). Then A^{-1} B_po^T ~ P^{-T/2} Q T^{-1} Q^T P^{-1/2} B_po^T and
    diag(Omega_p) ~ D_p + diag(B_po P^{-T/2} Q T^{-1} Q^T P^{-1/2} B_po^T).
Preconditioner 1 (P_L1 = B^T (W + D^{-1}) B): P^{-1/2} = S^{1/2} B^{-T} with
S = (W + D^{-1})^{-1}, so P^{-T/2} = B^{-1} S^{1/2}.
Preconditioner 2 (P_L2 = diag(Sigma_tilde + W^{-1})) is applied to the form-2 matrix
Sigma_tilde + W^{-1}: with G = Sigma_tilde + W^{-1} ~ P^{1/2} Q T Q^T P^{T/2},
A^{-1} B_po^T = W^{-1} G^{-1} Sigma_tilde B_po^T ~ W^{-1} P^{-1/2} Q T^{-1} Q^T P^{-1/2} Sigma_tilde B_po^T.
At k = n the factorisation is exact and so are the variances.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import laplace


def lanczos_basis(M_apply, v0: np.ndarray, k: int):
    """k steps (fewer if the Krylov space closes) of Lanczos with full
    reorthogonalisation. Returns (Q, T)."""
    n = len(v0)
    k = min(k, n)
    Q = np.zeros((n, k))
    Q[:, 0] = v0 / np.linalg.norm(v0)
    a, b = [], []
    for j in range(k):
        w = M_apply(Q[:, j])
        a.append(float(Q[:, j] @ w))
        for _ in range(2):
            w = w - Q[:, :j + 1] @ (Q[:, :j + 1].T @ w)
        nb = float(np.linalg.norm(w))
        if j + 1 == k or nb <= 1e-13 * max(abs(a[0]), 1e-300):
            Q = Q[:, :j + 1]
            break
        b.append(nb)
        Q[:, j + 1] = w / nb
    T = np.diag(a) + np.diag(b[: len(a) - 1], 1) + np.diag(b[: len(a) - 1], -1)
    return Q, T


def pred_var_lanczos(f: laplace.Factor, md: laplace.Mode, pf: laplace.PredFactor, k: int,
                     precond: int = 1) -> np.ndarray:
    W, D = md.W, f.D
    BpoT = pf.Bpo.toarray().T                          # (n, n_p) columns of B_po^T
    v = BpoT.mean(axis=1)
    Binv = lambda x: sla.solve_triangular(f.B.toarray(), x, lower=True, unit_diagonal=True)
    BinvT = lambda x: sla.solve_triangular(f.B.toarray().T, x, lower=False, unit_diagonal=True)
    if precond == 1:
        s = np.sqrt(1.0 / (W + 1.0 / D))               # S^{1/2}
        A = sp.diags(W) + f.Sinv
        Ph = lambda x: (s * BinvT(x).T).T if x.ndim == 2 else s * BinvT(x)     # P^{-1/2}
        PhT = lambda x: Binv((s * x.T).T) if x.ndim == 2 else Binv(s * x)     # P^{-T/2}
        M = lambda x: Ph(A @ PhT(x))
        Q, T = lanczos_basis(M, Ph(v), k)
        Y = Q.T @ Ph(BpoT)                             # (k, n_p)
        X = PhT(Q @ np.linalg.solve(T, Y))             # ~ A^{-1} B_po^T
    else:
        St = np.linalg.inv(f.Sinv.toarray())           # Sigma_tilde (small n)
        G = St + np.diag(1.0 / W)
        p = np.sqrt(np.diag(G))
        M = lambda x: (G @ (x / p)) / p
        StB = St @ BpoT
        Q, T = lanczos_basis(M, (St @ v) / p, k)
        Y = Q.T @ (StB / p[:, None])
        X = ((Q @ np.linalg.solve(T, Y)) / p[:, None]) / W[:, None]
    return pf.Dp + np.sum(BpoT * X, axis=0)
