"""Checks of a full-size run (the n = 1e6 grid workload, 359 levels) that the CPU oracle can
make at that size: outputs it computes one by one, and properties that hold at any size.

* neighbour sets and factor rows of sampled rows (brute-force neighbours, dense m x m
  solves; Section 2.1);
* the level recurrences on every row: lev(i) = 1 + max_{j in N(i)} lev(j) (0 without
  neighbours), and backward lev'(j) = 1 + max_{i: j in N(i)} lev'(i);
* stationarity of the mode (Eq. newton): grad psi(b) = d log p(y | F + b) - B^T D^{-1} B b
  is the residual of the last Newton system, so ||grad psi|| <= cg_tol ||W b + d log p||
  up to second-order terms;
* the assembly of L^VLA (Eq. VLA_loss) with the split log-determinant (Eq. logdetsplit,
  VADU): L = -sum log p + 1/2 sum_i (Bb)_i^2 / D_i + 1/2 (sum log D + sum log(W + 1/D) + mean gamma);
* Theorem 3.1's lower bound on each SLQ term: with ||r||^2 = n, gamma_i / n >= log of the
  smallest eigenvalue of the preconditioned matrix >= -log max_i (D_i W_ii + 1).

Test infrastructure: it takes the library's exported arrays (Vecchia order) as plain numpy
and uses only the oracle's definitions.
"""
from __future__ import annotations

import types

import numpy as np
import scipy.sparse as sp

from oracle import geometry, laplace as la, vecchia


def sample_rows(n: int, m: int, count: int, seed: int) -> np.ndarray:
    """The first rows (fewer than m predecessors, then the first full ones), `count` random
    rows and the last rows."""
    rng = np.random.default_rng(seed)
    head = np.arange(min(n, 2 * m + 2))
    tail = np.arange(max(0, n - 8), n)
    mid = rng.choice(n, size=min(n, count), replace=False)
    return np.unique(np.concatenate([head, mid, tail]))


def factor_rows(locs_v: np.ndarray, rows: np.ndarray, m: int, cov: int, sigma2: float, rho: float,
                nugget: float):
    """(N, A, D) of the given rows by the oracle's definitions. The factor rows are formed
    on a local table holding the sampled rows' own locations first and every location after
    them, so each row sees exactly its own neighbours."""
    N = geometry.knn_prev_rows(locs_v, m, rows)
    R = len(rows)
    loc_local = np.concatenate([locs_v[rows], locs_v])
    N_local = np.where(N >= 0, N + R, -1).astype(np.int64)
    A, D = vecchia.vecchia_factor(loc_local, N_local, cov, sigma2, rho, nugget)
    return N, A, D


def level_recurrences_hold(N: np.ndarray, lev_f: np.ndarray, lev_b: np.ndarray) -> tuple[bool, bool]:
    n, m = N.shape
    if m == 0:
        return bool(np.all(lev_f == 0)), bool(np.all(lev_b == 0))
    valid = N >= 0
    nb = np.where(valid, lev_f[np.where(valid, N, 0)], -1)
    ok_f = np.array_equal(lev_f, nb.max(1) + 1)
    best = np.full(n, -1, np.int64)
    rows = np.repeat(np.arange(n), m)[valid.ravel()]
    np.maximum.at(best, N.ravel()[valid.ravel()].astype(np.int64), lev_b[rows].astype(np.int64))
    ok_b = np.array_equal(lev_b, best + 1)
    return bool(ok_f), bool(ok_b)


def stationarity(N, A, D, y_v, F_v, b_v, lik: int, xi: float = 1.0) -> tuple[float, float]:
    """(||grad psi(b)||_2, ||W b + d log p||_2) at b (Vecchia order)."""
    B = vecchia.B_matrix(N, A)
    mu = F_v + b_v
    dlogp = la.grad_lik(y_v, mu, lik, xi)
    g = dlogp - B.T @ ((B @ b_v) / D)
    rhs = la.W_lik(y_v, mu, lik, xi) * b_v + dlogp
    return float(np.linalg.norm(g)), float(np.linalg.norm(rhs))


def lml_from_parts(N, A, D, y_v, F_v, b_v, lik: int, slq_mean: float, xi: float = 1.0) -> tuple[float, float]:
    """(L^VLA, log det(Sigma_tilde W + I)) assembled from the factor, the mode and the mean
    SLQ term, with the VADU split; b^T Sigma_tilde^{-1} b = sum (Bb)^2 / D without forming
    Sigma_tilde^{-1}."""
    B = vecchia.B_matrix(N, A)
    mu = F_v + b_v
    W = la.W_lik(y_v, mu, lik, xi)
    nll = -float(np.sum(la.log_lik(y_v, mu, lik, xi)))
    Bb = B @ b_v
    quad = 0.5 * float(np.sum(Bb * Bb / D))
    ld = float(np.sum(np.log(D))) + la.logdet_P(types.SimpleNamespace(D=D), W, la.PREC_VADU) + float(slq_mean)
    return nll + quad + 0.5 * ld, ld


def gamma_lower_bound(D, W) -> float:
    """Theorem 3.1 (VADU): every eigenvalue of P^{-1/2} A P^{-T/2} is at least
    min_i (D_i W_ii + 1)^{-1}, so gamma_i / n is at least the log of it."""
    return -float(np.log(np.max(D * W + 1.0)))


def solve_backward_error(N, A, X, Y, transpose: bool = False) -> float:
    """Componentwise backward error of a unit-triangular solve Y = B^{-1} X (or B^{-T} X):
    max over entries of |X - M Y| / (|X| + |M_off| |Y|), M = B or B^T. A substitution in a
    precision with unit roundoff u keeps it below gamma_k (rows of at most k terms; Higham,
    Accuracy and Stability of Numerical Algorithms, Thm 8.5), whatever the size."""
    B = vecchia.B_matrix(N, A)
    M = (B.T if transpose else B).tocsr()
    off = abs(M - sp.identity(M.shape[0], format="csr"))
    res = np.abs(X - M @ Y)
    scale = np.abs(X) + off @ np.abs(Y)
    return float(np.max(res / np.maximum(scale, np.finfo(float).tiny)))


def max_row_terms(N, transpose: bool = False) -> int:
    """Terms of the longest row of B (m + 1) or of B^T (1 + most dependents of one point)."""
    valid = N >= 0
    if not transpose:
        return int(valid.sum(1).max(initial=0)) + 1
    cnt = np.bincount(N[valid].ravel(), minlength=N.shape[0])
    return int(cnt.max(initial=0)) + 1
