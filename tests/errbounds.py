"""Rounding-error bounds for the operators of the Krylov path (test infrastructure).

Every GPU operator result is compared element by element with the float64 oracle under a
bound derived from the arithmetic instead of a fixed tolerance. u is the unit roundoff of
the working precision (2^-53 float64, 2^-24 float32) and gamma_k = k u / (1 - k u)
(Higham, Accuracy and Stability of Numerical Algorithms, 2nd ed., Sec. 3.1).

* A row of a product with B (one diagonal entry and at most m off-diagonal weights) is a
  dot product of at most m + 1 terms: |fl(BX) - BX| <= gamma_{m+1} |B| |X| (Sec. 3.1).
  Inputs and weights rounded to the working precision add u |B| |X| each.
* A unit triangular solve by substitution in any summation order has componentwise
  backward error |X - B Y_hat| <= gamma_{m+1} (|X| + |B_off| |Y_hat|) (Thm 8.5), hence the
  forward error |Y_hat - Y| <= |B^{-1}| gamma_{m+1} (|X| + |B_off| |Y_hat|).
* A diagonal scaling adds one rounding of the product and one of the scale.

The bounds are first order in u; the tests allow a factor 2 over them (BOUND_SLACK).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

U64 = 2.0 ** -53
U32 = 2.0 ** -24
BOUND_SLACK = 2.0


def gamma(k: int, u: float) -> float:
    return k * u / (1.0 - k * u)


def abs_parts(B: sp.spmatrix):
    """|B| and |B_off| (the strictly lower part) of a unit lower-triangular B."""
    aB = abs(B).tocsr()
    off = (aB - sp.identity(B.shape[0], format="csr")).tocsr()
    off.eliminate_zeros()
    return aB, off


def row_terms(off) -> int:
    """Most terms in one row's dot product: the diagonal plus the row's off-diagonal entries."""
    return int(np.diff(off.indptr).max(initial=0)) + 1


def product_bound(aB, X, k: int, u: float) -> np.ndarray:
    """|fl(B X) - B X| for rows of at most k terms, inputs and weights stored in the working
    precision."""
    return (gamma(k, u) + 2 * u) * (aB @ np.abs(X))


def solve_bound(aBinv: np.ndarray, off, X, Yhat, k: int, u: float) -> np.ndarray:
    """|Y_hat - B^{-1} X| for a substitution in the working precision with rows of at most k
    terms (X and the weights rounded to it first): |B^{-1}| (gamma_k + 2u)(|X| + |B_off| |Y_hat|)."""
    r = (gamma(k, u) + 2 * u) * (np.abs(X) + off @ np.abs(Yhat))
    return aBinv @ r


def scaled_solve_bound(aBinv, off, s, Y1, e1, Zhat, k: int, u: float) -> np.ndarray:
    """Z = B^{-1} (s o Y1) where Y1 carries the error bound e1 and s is rounded to the
    working precision: the propagated part |B^{-1}| (|s| e1 + 2u |s| |Y1|) plus the rounding of
    the solve itself."""
    S = np.abs(s)[:, None] if Y1.ndim == 2 else np.abs(s)
    Y2 = S * np.abs(Y1)
    prop = aBinv @ (S * e1 + 2 * u * Y2)
    own = (gamma(k, u) + 2 * u) * (Y2 + off @ np.abs(Zhat))
    return prop + aBinv @ own


def operator_bounds(B, D, W, dsc, X, Y: dict, ops: dict, u: float) -> dict:
    """Bounds for every operator of vl_apply given the computed results Y[op] (Vecchia order,
    float64 copies of the GPU results) and the exact reference solutions needed inside
    compositions. ops maps names to the library's op codes. Rows of B have at most m + 1
    terms; rows of B^T as many as the most-used neighbour has dependents, plus one."""
    Bd = B.toarray()
    aB, off = abs_parts(B)
    aBt, offt = aB.T.tocsr(), off.T.tocsr()
    kf, kb = row_terms(off), row_terms(offt)
    aBinv = np.abs(np.linalg.inv(Bd))
    aBtinv = aBinv.T
    absX = np.abs(X)
    col = (lambda v: v[:, None]) if X.ndim == 2 else (lambda v: v)
    out = {}
    out[ops["B"]] = product_bound(aB, X, kf, u)
    out[ops["BT"]] = product_bound(aBt, X, kb, u)
    # A X = W X + B^T (D^{-1} o (B X)): the inner product, its scaling, then the outer product
    # (one more term per row: W X)
    BX = Bd @ X
    e_in = product_bound(aB, X, kf, u)
    Yin = col(1.0 / D) * BX
    e_y = col(1.0 / D) * e_in + 2 * u * np.abs(Yin)
    out[ops["A"]] = (col(np.abs(W)) * absX * 3 * u + aBt @ e_y
                     + (gamma(kb + 1, u) + 2 * u) * (aBt @ np.abs(Yin) + col(np.abs(W)) * absX))
    out[ops["BINV"]] = solve_bound(aBinv, off, X, Y[ops["BINV"]], kf, u)
    out[ops["BTINV"]] = solve_bound(aBtinv, offt, X, Y[ops["BTINV"]], kb, u)
    # Sigma X = B^{-1} (D o B^{-T} X) and P^{-1} X = B^{-1} (dsc o B^{-T} X); Y1 = B^{-T} X
    Y1 = np.linalg.solve(Bd.T, X)
    e1 = solve_bound(aBtinv, offt, X, Y[ops["BTINV"]], kb, u)
    out[ops["SIGMA"]] = scaled_solve_bound(aBinv, off, D, Y1, e1, Y[ops["SIGMA"]], kf, u)
    out[ops["PINV"]] = scaled_solve_bound(aBinv, off, dsc, Y1, e1, Y[ops["PINV"]], kf, u)
    # (Sigma + W^{-1}) X: the Sigma part, the rounded W^{-1} o X and the final sum
    out[ops["A2"]] = (out[ops["SIGMA"]] + 3 * u * col(1.0 / np.abs(W)) * absX
                      + u * np.abs(Y[ops["A2"]]))
    return out
