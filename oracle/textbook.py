"""Dense GP Laplace approximation in the covariance parametrisation.

This is the standard textbook route (Rasmussen & Williams, "Gaussian Processes
for Machine Learning", 2006, Algorithms 3.1 and 3.2, written for a general
log-concave likelihood with diagonal W). It never forms a precision matrix or a
Vecchia factor, so it is an independent check of the Vecchia-Laplace oracle in
the case where the Vecchia approximation is exact (m = n - 1 for training,
every training point as neighbour of each prediction point).

    f <- 0;  repeat: W = -grad^2 log p(y | F + f);  L = chol(I + W^1/2 K W^1/2)
             b = W f + grad log p;  a = b - W^1/2 L^T \\ (L \\ (W^1/2 K b));  f = K a
    -log q(y) = 1/2 a^T f - log p(y | F + f) + sum log L_ii
    predictive mean  F_p + k_*^T grad log p(y | F + f)
    predictive var   k_** - v^T v,  v = L \\ (W^1/2 k_*)
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import laplace


def gp_laplace(K: np.ndarray, y: np.ndarray, F: np.ndarray, lik: int, tol=1e-13, max_iter=200, xi: float = 1.0):
    n = len(y)
    f = np.zeros(n)
    for _ in range(max_iter):
        mu = F + f
        W = laplace.W_lik(y, mu, lik, xi)
        sW = np.sqrt(W)
        L = np.linalg.cholesky(np.eye(n) + sW[:, None] * K * sW[None, :])
        bb = W * f + laplace.grad_lik(y, mu, lik, xi)
        rhs = sW * (K @ bb)
        a = bb - sW * sla.solve_triangular(L.T, sla.solve_triangular(L, rhs, lower=True), lower=False)
        f_new = K @ a
        done = np.max(np.abs(f_new - f)) <= tol * (1.0 + np.max(np.abs(f_new)))
        f = f_new
        if done:
            break
    mu = F + f
    W = laplace.W_lik(y, mu, lik, xi)
    sW = np.sqrt(W)
    L = np.linalg.cholesky(np.eye(n) + sW[:, None] * K * sW[None, :])
    a = np.linalg.solve(K, f)
    nlml = 0.5 * a @ f - np.sum(laplace.log_lik(y, mu, lik, xi)) + np.sum(np.log(np.diag(L)))
    return f, float(nlml), L, W


def gp_predict(K: np.ndarray, Ks: np.ndarray, kss: np.ndarray, y, F, Fp, f, L, W, lik, xi: float = 1.0):
    """Ks: (n, n_p) cross covariances, kss: (n_p,) prior variances at test points."""
    g = laplace.grad_lik(y, F + f, lik, xi)
    mean = np.asarray(Fp, float) + Ks.T @ g
    v = sla.solve_triangular(L, np.sqrt(W)[:, None] * Ks, lower=True)
    return mean, kss - np.sum(v * v, axis=0)
