"""Neighbour sets and level schedules, by brute force and by definition.

Section 2.1: N(i) is a subset of {1, ..., i-1} with |N(i)| <= m; for i > m + 1 it
is the m nearest neighbours of s_i among s_1, ..., s_{i-1}. Read here (0-based):
N(i) = the min(i, m) points j < i with the smallest key (d2_ij, j), listed in
ascending key order, where d2 = (xi - xj)*(xi - xj) + (yi - yj)*(yi - yj) is
evaluated in float64, left to right, each operation rounded (no fused
multiply-add). Unused slots hold -1.

Section 4.1: prediction points condition only on observed points; their
neighbour sets are the m nearest training points under the same key.

Level schedules of the unit lower-triangular B (rows depend on N(i)):
lev(i)  = 0 if N(i) is empty, else 1 + max_{j in N(i)} lev(j)      (forward)
levT(j) = 0 if no row lists j, else 1 + max_{i : j in N(i)} levT(i)  (backward)
"""
from __future__ import annotations

import numpy as np


def _d2(x, y, xs, ys):
    dx = x - xs
    dy = y - ys
    return dx * dx + dy * dy   # numpy: each op separately rounded, no contraction


def _select(d2: np.ndarray, idx: np.ndarray, k: int) -> np.ndarray:
    """The k smallest (d2, idx) keys in ascending order (exact on ties)."""
    if k <= 0:
        return np.zeros(0, np.int64)
    if len(d2) > k:
        kth = np.partition(d2, k - 1)[k - 1]
        keep = d2 <= kth
        d2, idx = d2[keep], idx[keep]
    o = np.lexsort((idx, d2))
    return idx[o[:k]]


def knn_prev_rows(locs: np.ndarray, m: int, rows) -> np.ndarray:
    """N(i) for the requested rows i (locations already in Vecchia order)."""
    x, y = locs[:, 0], locs[:, 1]
    rows = np.asarray(rows, dtype=np.int64)
    out = np.full((len(rows), m), -1, np.int32)
    for a, i in enumerate(rows):
        k = min(int(i), m)
        if k == 0:
            continue
        d2 = _d2(x[i], y[i], x[:i], y[:i])
        out[a, :k] = _select(d2, np.arange(i), k)
    return out


def knn_prev(locs: np.ndarray, m: int) -> np.ndarray:
    """N(i) for every row; O(n^2), intended for n up to a few 10^4."""
    return knn_prev_rows(locs, m, np.arange(len(locs)))


def knn_cross(train: np.ndarray, test: np.ndarray, m: int) -> np.ndarray:
    """The min(m, n) nearest training points (by (d2, training index)) of each test point."""
    n = len(train)
    k = min(m, n)
    out = np.full((len(test), m), -1, np.int32)
    for a in range(len(test)):
        d2 = _d2(test[a, 0], test[a, 1], train[:, 0], train[:, 1])
        out[a, :k] = _select(d2, np.arange(n), k)
    return out


def levels_forward(N: np.ndarray) -> np.ndarray:
    n = N.shape[0]
    lev = np.zeros(n, np.int32)
    for i in range(n):
        nb = N[i][N[i] >= 0]
        lev[i] = 1 + lev[nb].max() if len(nb) else 0
    return lev


def levels_backward(N: np.ndarray) -> np.ndarray:
    n = N.shape[0]
    levT = np.zeros(n, np.int32)
    for i in range(n - 1, -1, -1):
        for j in N[i][N[i] >= 0]:
            if levT[i] + 1 > levT[j]:
                levT[j] = levT[i] + 1
    return levT
