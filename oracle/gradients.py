"""Gradients of L^VLA with respect to the covariance parameters theta = (sigma2, rho),
exactly and by stochastic trace estimation (STE, Eq. grad_STE) with the control
variate of Section 3, for the VADU preconditioner. Test infrastructure: a plain
float64 CPU restatement of the paper (appendix "Gradients of Vecchia-Laplace
approximations", "Derivatives of log-determinants using stochastic trace estimation
and variance reduction", "Derivatives of the Vecchia-approximated precision and
covariance matrices"); nothing here is used by the CUDA path.

The nugget follows the shared reading tau = ratio * sigma2 (ratio = nugget / sigma2 of
the factor, 1e-10 by default), so Sigma = sigma2 (R(rho) + ratio I) and
    d Sigma / d sigma2 = Sigma / sigma2,     d Sigma / d rho = sigma2 dR / d rho.
Covariance derivatives in rho: exponential sigma2 e^{-h/rho} h / rho^2; Matern-1.5
sigma2 a^2 e^{-a} / rho with a = sqrt(3) h / rho.

Vecchia factor (row i, N = N(i), A_i = Sigma_{i,N} Sigma_N^{-1}):
    dA_i = (dSigma_{i,N} - A_i dSigma_N) Sigma_N^{-1}
    dD_i = dSigma_ii - dA_i Sigma_{N,i} - A_i dSigma_{N,i}
    dB_{i,N} = -dA_i
    d Sigma_tilde^{-1} = dB^T D^{-1} B + B^T D^{-1} dB - B^T D^{-1} dD D^{-1} B
Gradient in the offset F (same appendix; db*/dF_i = -A^{-1} W e_i):
    dL/dF = -grad log p(y | mu*) + g - W o (A^{-1} g).
Exact gradient (A = W + Sigma_tilde^{-1}, b* the mode, W'_i = dW_ii / d mu_i):
    dL/dtheta = 1/2 b*^T dSinv b* + 1/2 [sum_i dD_i / D_i + tr(A^{-1} dSinv)]
                - (A^{-1} g)^T dSinv b*,    g_i = dL / db*_i = 1/2 (A^{-1})_ii W'_i,
the last term being the implicit one, (dL/db*)^T db*/dtheta with
db*/dtheta = -A^{-1} dSinv b*.
STE (probes z with E z z^T = P, P = B^T (W + D^{-1}) B):
    d logdet(Sigma_tilde W + I)/dtheta ~ sum dD_i/D_i - c tr((W + D^{-1})^{-1} D^{-1} dD D^{-1})
                                        + mean_i [h(z_i) - c r(z_i)]
    h(z) = (A^{-1} z)^T dSinv P^{-1} z
    r(z) = (P^{-1} z)^T (dSinv + dB^T W B + B^T W dB) P^{-1} z    (= z^T P^{-1} dP P^{-1} z)
    d logdet/d mu_j ~ c_j (W + D^{-1})^{-1}_jj W'_j + mean_i [h_j(z_i) - c_j r_j(z_i)],
    h_j(z) = (A^{-1} z)_j W'_j (P^{-1} z)_j,  r_j(z) = (B P^{-1} z)_j^2 W'_j,
with c = Cov(h, r) / Var(r) over the probes (c = 0: plain STE).
Auxiliary likelihood parameter xi (gamma shape alpha; same appendix), with
dW/dxi = -d^3 log p / dxi dmu^2 and db*/dxi = A^{-1} d^2 log p / dxi dmu:
    dL/dxi = -sum_i d log p_i / dxi + 1/2 tr(A^{-1} dW/dxi) + (A^{-1} g)^T d^2 log p / dxi dmu,
    STE: d logdet / dxi ~ c tr((W + D^{-1})^{-1} dW/dxi) + mean_i [h(z_i) - c r(z_i)],
         h(z) = (A^{-1} z)^T dW/dxi P^{-1} z,   r(z) = (B P^{-1} z)^T dW/dxi (B P^{-1} z).
Linear fixed effects F = X beta (Section 2): dL/dbeta = X^T dL/dF.
LRAC form (appendix, "Preconditioner LRAC"; P = L_k L_k^T + W^{-1}, probes z = L_k r1 +
W^{-1/2} r2, form-2 matrix Sigma_tilde + W^{-1}). With the pivot set I fixed, the rank-k
pivoted Cholesky factor satisfies L_k L_k^T = Sigma_{:,I} Sigma_{I,I}^{-1} Sigma_{I,:}, so
    d(L_k L_k^T) = dS_{:,I} G + G^T dS_{I,:} - G^T dS_{I,I} G,   G = Sigma_{I,I}^{-1} Sigma_{I,:},
and the control variate's mean is tr(P^{-1} d(L_k L_k^T)) = d log det P:
    d logdet / d theta ~ c tr(P^{-1} d(LL^T)) + mean_i [h(z_i) - c r(z_i)],
        h(z) = -((Sigma_tilde + W^{-1})^{-1} z)^T Sigma_tilde dSinv Sigma_tilde P^{-1} z,
        r(z) = (P^{-1} z)^T d(LL^T) P^{-1} z;
    d logdet / d mu_j ~ W'_j / W_j + c_j (W'_j (L C^{-1} L^T)_jj - W'_j / W_j) - mean_i [h_j - c_j r_j],
        h_j(z) = ((Sigma_tilde + W^{-1})^{-1} z)_j W'_j / W_j^2 (P^{-1} z)_j,
        r_j(z) = (P^{-1} z)_j^2 W'_j / W_j^2,       C = I_k + L^T W L,
using (Sigma_tilde + W^{-1})^{-1} = W A^{-1} Sigma_tilde^{-1}. When the control
variate is constant over the probes its variance is rounding noise and c is set to 0:
with Rademacher probes and VADU this happens for sigma2 (B does not depend on sigma2
and r(z) = -sum_i (W_i + 1/D_i)^{-1} / (sigma2 D_i) for every z), where Cov / Var would
multiply rounding differences by a huge weight.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
from scipy.special import digamma

from . import laplace, lrac, vecchia

PARAMS = ("sigma2", "rho")


def W_prime(y, mu, lik, xi: float = 1.0):
    """dW/dmu = -d^3 log p / d mu^3 (W = -d^2 log p / d mu^2)."""
    if lik == laplace.LIK_BERNOULLI_LOGIT:
        p = 1.0 / (1.0 + np.exp(-mu))
        return p * (1.0 - p) * (1.0 - 2.0 * p)
    if lik == laplace.LIK_GAMMA_LOG:
        return -float(xi) * y * np.exp(-mu)
    return np.exp(mu)


# gamma, u = y e^{-mu}:  d log p / d alpha = log alpha + 1 - digamma(alpha) + log y - mu - u,
# d^2 log p / d alpha d mu = u - 1,   dW / d alpha = u.
def dloglik_dxi(y, mu, lik, xi):
    _gamma_only(lik)
    return np.log(xi) + 1.0 - digamma(xi) + np.log(y) - mu - y * np.exp(-mu)


def d2loglik_dxi_dmu(y, mu, lik, xi):
    _gamma_only(lik)
    return y * np.exp(-mu) - 1.0


def dW_dxi(y, mu, lik, xi):
    _gamma_only(lik)
    return y * np.exp(-mu)


def _gamma_only(lik):
    if lik != laplace.LIK_GAMMA_LOG:
        raise ValueError("only the gamma likelihood has an auxiliary parameter")


def dcov(h, cov, sigma2, rho, param, nugget_ratio, same_point):
    """d Sigma_{uv} / d theta for distances h; same_point marks u = v (nugget)."""
    if param == "sigma2":
        return vecchia.cov_fn(h, cov, 1.0, rho) + np.where(same_point, nugget_ratio, 0.0)
    if cov == vecchia.COV_EXPONENTIAL:
        return sigma2 * np.exp(-h / rho) * h / (rho * rho)
    a = math.sqrt(3.0) * h / rho
    return sigma2 * a * a * np.exp(-a) / rho


def factor_derivatives(f: laplace.Factor, param: str):
    """(dA, dD) aligned with f.N / f.D, rows batched by neighbour count."""
    n, m = f.N.shape
    ratio = f.nugget / f.sigma2
    dA = np.zeros((n, m))
    dD = np.empty(n)
    k_of = (f.N >= 0).sum(1)
    for k in range(m + 1):
        rows = np.nonzero(k_of == k)[0]
        if len(rows) == 0:
            continue
        dii = dcov(np.zeros(len(rows)), f.cov, f.sigma2, f.rho, param, ratio, True)
        if k == 0:
            dD[rows] = dii
            continue
        nb = f.N[rows, :k]
        P = f.locs[nb]
        hNN = vecchia.dist(P[:, :, None, :], P[:, None, :, :])
        same = np.broadcast_to(np.eye(k, dtype=bool), hNN.shape)
        S_NN = vecchia.cov_fn(hNN, f.cov, f.sigma2, f.rho)
        S_NN[:, np.arange(k), np.arange(k)] += f.nugget
        dS_NN = dcov(hNN, f.cov, f.sigma2, f.rho, param, ratio, same)
        hNi = vecchia.dist(P, f.locs[rows][:, None, :])
        S_Ni = vecchia.cov_fn(hNi, f.cov, f.sigma2, f.rho)
        dS_Ni = dcov(hNi, f.cov, f.sigma2, f.rho, param, ratio, np.zeros_like(hNi, dtype=bool))
        Ai = f.A[rows, :k]
        # dA_i = (dSigma_{i,N} - A_i dSigma_N) Sigma_N^{-1}   (Sigma_N symmetric)
        rhs = dS_Ni - np.einsum("rk,rkl->rl", Ai, dS_NN)
        dAi = np.linalg.solve(S_NN, rhs[..., None])[..., 0]
        dA[rows, :k] = dAi
        dD[rows] = dii - (dAi * S_Ni).sum(1) - (Ai * dS_Ni).sum(1)
    return dA, dD


def dB_matrix(f: laplace.Factor, dA) -> sp.csr_matrix:
    n, m = f.N.shape
    rows = np.repeat(np.arange(n), m)
    cols = f.N.ravel()
    ok = cols >= 0
    return sp.csr_matrix((-dA.ravel()[ok], (rows[ok], cols[ok])), shape=(n, n))


def dSinv_matrix(f: laplace.Factor, dB, dD) -> sp.csr_matrix:
    Dinv = sp.diags(1.0 / f.D)
    return (dB.T @ Dinv @ f.B + f.B.T @ Dinv @ dB - f.B.T @ sp.diags(dD / (f.D * f.D)) @ f.B).tocsr()


def lml_grad_exact(f: laplace.Factor, md: laplace.Mode) -> dict:
    """dL^VLA / d theta by the formulas above with dense A^{-1} (small n only)."""
    A = np.diag(md.W) + f.Sinv.toarray()
    Ainv = np.linalg.inv(A)
    g = 0.5 * np.diag(Ainv) * W_prime(md.y, md.mu, md.lik, md.xi)
    Ag = Ainv @ g
    out = {}
    for par in PARAMS:
        dA, dD = factor_derivatives(f, par)
        dS = dSinv_matrix(f, dB_matrix(f, dA), dD)
        dSb = dS @ md.b
        logdet_part = float(np.sum(dD / f.D) + np.sum(Ainv * dS.toarray()))
        out[par] = 0.5 * float(md.b @ dSb) + 0.5 * logdet_part - float(Ag @ dSb)
    return out


def lml_grad_F_exact(f: laplace.Factor, md: laplace.Mode) -> np.ndarray:
    """dL^VLA / dF in caller order (dense A^{-1}, small n only)."""
    Ainv = np.linalg.inv(np.diag(md.W) + f.Sinv.toarray())
    g = 0.5 * np.diag(Ainv) * W_prime(md.y, md.mu, md.lik, md.xi)
    dF = -laplace.grad_lik(md.y, md.mu, md.lik, md.xi) + g - md.W * (Ainv @ g)
    out = np.empty(f.n)
    out[f.order] = dF
    return out


def lml_grad_xi_exact(f: laplace.Factor, md: laplace.Mode) -> float:
    """dL^VLA / dxi (gamma shape) with dense A^{-1} (small n only)."""
    Ainv = np.linalg.inv(np.diag(md.W) + f.Sinv.toarray())
    g = 0.5 * np.diag(Ainv) * W_prime(md.y, md.mu, md.lik, md.xi)
    explicit = -float(np.sum(dloglik_dxi(md.y, md.mu, md.lik, md.xi)))
    logdet = float(np.sum(np.diag(Ainv) * dW_dxi(md.y, md.mu, md.lik, md.xi)))
    implicit = float((Ainv @ g) @ d2loglik_dxi_dmu(md.y, md.mu, md.lik, md.xi))
    return explicit + 0.5 * logdet + implicit


def lml_grad_beta(X, dF) -> np.ndarray:
    """dL^VLA / dbeta = X^T dL/dF for F = X beta (X n x p and dF in caller order)."""
    return np.asarray(X, float).T @ np.asarray(dF, float)


def _solvers(f: laplace.Factor, W):
    lo, up = laplace._tri_solvers(f.B)          # B^{-1} and B^{-T}
    A_lu = laplace._lu(sp.diags(W) + f.Sinv)
    s = 1.0 / (W + 1.0 / f.D)                   # (W + D^{-1})^{-1}
    P_inv = lambda Z: np.column_stack([lo(s * up(Z[:, j])) for j in range(Z.shape[1])])
    return A_lu, P_inv


def lml_grad_ste(f: laplace.Factor, md: laplace.Mode, t: int, seed: int, control_variate: bool = True) -> dict:
    """dL^VLA / d theta with every log-determinant derivative by STE on the same t
    Rademacher probes z = P^{1/2} r (VADU); the implicit term solves A once for
    A^{-1} g. Returns the gradient and, per parameter, the samples h and r."""
    W, Wp = md.W, W_prime(md.y, md.mu, md.lik, md.xi)
    R = laplace.probes(f, t, seed)
    Z = f.B.T @ (np.sqrt(W + 1.0 / f.D)[:, None] * R)          # z = P^{1/2} r
    A_lu, P_inv = _solvers(f, W)
    AZ = A_lu.solve(Z)                                          # A^{-1} z
    PZ = P_inv(Z)                                               # P^{-1} z
    BPZ = f.B @ PZ
    # d logdet / d mu_j for the implicit term
    hj = AZ * Wp[:, None] * PZ
    rj = BPZ * BPZ * Wp[:, None]
    if control_variate and t > 1:
        vr = rj.var(axis=1, ddof=1)
        live = vr > 1e-20 * rj.mean(1) ** 2
        cj = np.where(live, ((hj - hj.mean(1, keepdims=True)) * (rj - rj.mean(1, keepdims=True))).sum(1)
                      / (t - 1) / np.where(live, vr, 1.0), 0.0)
    else:
        cj = np.zeros(f.n)
    dld_dmu = cj * Wp / (W + 1.0 / f.D) + (hj - cj[:, None] * rj).mean(1)
    g = 0.5 * dld_dmu
    Ag = A_lu.solve(g)
    dF = np.empty(f.n)
    dF[f.order] = -laplace.grad_lik(md.y, md.mu, md.lik, md.xi) + g - W * Ag
    out, samples = {"F": dF}, {}
    if md.lik == laplace.LIK_GAMMA_LOG:
        dW = dW_dxi(md.y, md.mu, md.lik, md.xi)
        h = np.einsum("ij,ij->j", AZ, dW[:, None] * PZ)
        r = np.einsum("ij,ij->j", BPZ, dW[:, None] * BPZ)
        c = 0.0
        if control_variate and t > 1 and r.var(ddof=1) > 1e-20 * r.mean() ** 2:
            c = float(np.cov(h, r, ddof=1)[0, 1] / r.var(ddof=1))
        dlogdet = c * float(np.sum(dW / (W + 1.0 / f.D))) + float(np.mean(h - c * r))
        d2 = d2loglik_dxi_dmu(md.y, md.mu, md.lik, md.xi)
        out["xi"] = (-float(np.sum(dloglik_dxi(md.y, md.mu, md.lik, md.xi))) + 0.5 * dlogdet
                     + float(Ag @ d2))
        w = A_lu.solve(d2)
        per_probe = 0.5 * (h - c * r) + 0.5 * (w[:, None] * (hj - cj[:, None] * rj)).sum(0)
        samples["xi"] = {"h": h, "r": r, "c": c, "dlogdet": dlogdet, "per_probe": per_probe}
    for par in PARAMS:
        dA, dD = factor_derivatives(f, par)
        dB = dB_matrix(f, dA)
        dS = dSinv_matrix(f, dB, dD)
        h = np.einsum("ij,ij->j", AZ, dS @ PZ)
        M = dS + dB.T @ sp.diags(W) @ f.B + f.B.T @ sp.diags(W) @ dB
        r = np.einsum("ij,ij->j", PZ, M @ PZ)
        c = 0.0
        if control_variate and t > 1 and r.var(ddof=1) > 1e-20 * r.mean() ** 2:
            c = float(np.cov(h, r, ddof=1)[0, 1] / r.var(ddof=1))
        tr_dlogP = -float(np.sum(dD / (f.D * f.D) / (W + 1.0 / f.D)))
        dlogdet = float(np.sum(dD / f.D)) + c * tr_dlogP + float(np.mean(h - c * r))
        dSb = dS @ md.b
        out[par] = 0.5 * float(md.b @ dSb) + 0.5 * dlogdet - float(Ag @ dSb)
        # per-probe contribution to the gradient (its spread gives the standard error):
        # 1/2 (h - c r) and, through g, -1/2 sum_j w_j (h_j - c_j r_j) with w = A^{-1} dSinv b*
        w = A_lu.solve(dSb)
        per_probe = 0.5 * (h - c * r) - 0.5 * (w[:, None] * (hj - cj[:, None] * rj)).sum(0)
        samples[par] = {"h": h, "r": r, "c": c, "dlogdet": dlogdet, "per_probe": per_probe}
    return {"grad": out, "samples": samples}


def dlogdet_exact(f: laplace.Factor, md: laplace.Mode) -> dict:
    """d log det(Sigma_tilde W + I) / d theta at fixed W: sum dD_i / D_i + tr(A^{-1} dSinv)."""
    Ainv = np.linalg.inv(np.diag(md.W) + f.Sinv.toarray())
    out = {}
    for par in PARAMS:
        dA, dD = factor_derivatives(f, par)
        dS = dSinv_matrix(f, dB_matrix(f, dA), dD)
        out[par] = float(np.sum(dD / f.D) + np.sum(Ainv * dS.toarray()))
    return out


# ----------------------------------------------------------------------------- LRAC form
def lowrank_derivative(f: laplace.Factor, piv, param: str) -> np.ndarray:
    """d(L_k L_k^T)/dtheta (dense n x n, Vecchia order) at the fixed pivot set piv."""
    piv = np.asarray(piv, np.int64)
    n = f.n
    ratio = f.nugget / f.sigma2
    h = vecchia.dist(f.locs[:, None, :], f.locs[piv][None, :, :])               # n x k
    same = np.arange(n)[:, None] == piv[None, :]
    S = vecchia.cov_fn(h, f.cov, f.sigma2, f.rho) + np.where(same, f.nugget, 0.0)
    dS = dcov(h, f.cov, f.sigma2, f.rho, param, ratio, same)
    G = np.linalg.solve(S[piv], S.T)                                            # Sigma_II^{-1} Sigma_I:
    return dS @ G + G.T @ dS.T - G.T @ dS[piv] @ G


def _cv_weight(h, r, t, control_variate):
    if control_variate and t > 1 and r.var(ddof=1) > 1e-20 * r.mean() ** 2:
        return float(np.cov(h, r, ddof=1)[0, 1] / r.var(ddof=1))
    return 0.0


def lml_grad_ste_lrac(f: laplace.Factor, md: laplace.Mode, k: int, t: int, seed: int,
                      control_variate: bool = True) -> dict:
    """dL^VLA / d theta and dL/dF with the log-determinant derivatives by STE on the LRAC
    probes (dense pieces: small n only). Same return layout as lml_grad_ste."""
    W, Wp = md.W, W_prime(md.y, md.mu, md.lik, md.xi)
    L, piv = lrac.pivoted_cholesky(f.locs, f.cov, f.sigma2, f.rho, f.nugget, k)
    Z = lrac.lrac_probes(f, L, W, t, seed)
    PZ = lrac.woodbury_apply(L, W, Z)                                   # P^{-1} z
    A_lu = laplace._lu(sp.diags(W) + f.Sinv)
    UZ = W[:, None] * A_lu.solve(f.Sinv @ Z)                            # (Sigma_tilde + W^{-1})^{-1} z
    C = np.eye(L.shape[1]) + L.T @ (W[:, None] * L)
    lo, up = laplace._tri_solvers(f.B)
    St = lambda V: np.column_stack([lo(f.D * up(V[:, j])) for j in range(V.shape[1])])   # Sigma_tilde V
    # d logdet / d mu_j (implicit term)
    q = Wp / (W * W)
    hj = UZ * q[:, None] * PZ
    rj = PZ * PZ * q[:, None]
    if control_variate and t > 1:
        vr = rj.var(axis=1, ddof=1)
        live = vr > 1e-20 * rj.mean(1) ** 2
        cj = np.where(live, ((hj - hj.mean(1, keepdims=True)) * (rj - rj.mean(1, keepdims=True))).sum(1)
                      / (t - 1) / np.where(live, vr, 1.0), 0.0)
    else:
        cj = np.zeros(f.n)
    diag_LCL = np.einsum("ij,ij->i", L, np.linalg.solve(C, L.T).T)
    trW = Wp / W
    dld_dmu = trW + cj * (Wp * diag_LCL - trW) - (hj - cj[:, None] * rj).mean(1)
    g = 0.5 * dld_dmu
    Ag = A_lu.solve(g)
    dF = np.empty(f.n)
    dF[f.order] = -laplace.grad_lik(md.y, md.mu, md.lik, md.xi) + g - W * Ag
    out, samples = {"F": dF}, {}
    StU, StP = St(UZ), St(PZ)
    for par in PARAMS:
        dA, dD = factor_derivatives(f, par)
        dS = dSinv_matrix(f, dB_matrix(f, dA), dD)
        h = -np.einsum("ij,ij->j", StU, dS @ StP)
        dLL = lowrank_derivative(f, piv, par)
        r = np.einsum("ij,ij->j", PZ, dLL @ PZ)
        c = _cv_weight(h, r, t, control_variate)
        tr_dlogP = float(np.trace(lrac.woodbury_apply(L, W, dLL)))      # tr(P^{-1} d(LL^T))
        dlogdet = c * tr_dlogP + float(np.mean(h - c * r))
        dSb = dS @ md.b
        out[par] = 0.5 * float(md.b @ dSb) + 0.5 * dlogdet - float(Ag @ dSb)
        w = A_lu.solve(dSb)
        per_probe = 0.5 * (h - c * r) + 0.5 * (w[:, None] * (hj - cj[:, None] * rj)).sum(0)
        samples[par] = {"h": h, "r": r, "c": c, "dlogdet": dlogdet, "per_probe": per_probe,
                        "tr_dlogP": tr_dlogP}
    samples["mu"] = {"h": hj, "r": rj, "c": cj, "dlogdet": dld_dmu}
    return {"grad": out, "samples": samples, "pivots": piv}
