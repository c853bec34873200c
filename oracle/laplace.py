"""Vecchia-Laplace quantities by direct methods (the "Cholesky-VL" analogue).

Model (Section 2): mu = F + b, b ~ N(0, Sigma_tilde), Sigma_tilde^{-1} = B^T D^{-1} B,
y_i | mu_i independent with a log-concave density.

Mode (Eq. newton):  b^{t+1} = (W + Sigma_tilde^{-1})^{-1} (W b^t + d log p / d b),
W = -d^2 log p / d mu^2 (diagonal). Readings shared with the CUDA side:
b^0 = 0; a step is halved (up to 30 times) while it lowers
psi(b) = log p(y | F + b) - 1/2 b^T Sigma_tilde^{-1} b by more than 1e-12 (1 + |psi|);
stop when max_i |b^{t+1}_i - b^t_i| <= newton_tol (1 + max_i |b^{t+1}_i|).
Each linear system is solved by a sparse LU factorisation (SuperLU).

L^VLA (Eq. VLA_loss) = -log p(y | mu*) + 1/2 b*^T Sigma_tilde^{-1} b*
                       + 1/2 log det(Sigma_tilde W + I).
log det(Sigma_tilde W + I) = sum_i log D_i + log det(W + Sigma_tilde^{-1})
(det B = 1), the second term from the diagonal of the sparse LU factor.
log p includes all constant terms (for Poisson, -log y!).

Same-probe SLQ (Eqs. logdetsplit, def_SLQ; Section 3.1.1):
log det(Sigma_tilde W + I) = sum log D_i + log det P + log det(P^{-1/2} A P^{-T/2}),
A = W + Sigma_tilde^{-1};  VADU P = B^T (W + D^{-1}) B, log det P = sum log(W_i + 1/D_i);
LVA P = B^T D^{-1} B, log det P = -sum log D_i. Probes z = P^{1/2} r with r
Rademacher, P^{1/2} = B^T (W + D^{-1})^{1/2} (VADU) or B^T D^{-1/2} (LVA), so
P^{-1/2} z = r and ||P^{-1/2} z||^2 = n exactly. Each gamma_i =
||r_i||^2 e1^T log(T_i) e1 comes from explicit Lanczos with full
reorthogonalisation on P^{-1/2} A P^{-T/2} started at r_i.

Prediction (Eq. latentpostpredictive, Section 4.1 ordering: observed points
first, each prediction point conditioned on m observed points only, so B_p = I):
omega_p = F_p - B_po b*,  Omega_p = D_p + B_po A^{-1} B_po^T  (diagonal only).
Algorithm simAlgo: z3 = W^{1/2} z1 + B^T D^{-1/2} z2, z4 = B_po A^{-1} z3,
var_p = D_p + (1/s) sum_k z4[p, k]^2.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import gammaln

from . import geometry, krylov, rng as orng, vecchia

LIK_BERNOULLI_LOGIT = 0
LIK_POISSON_LOG = 1
LIK_GAMMA_LOG = 2
PREC_VADU = 0
PREC_LVA = 1


# ----------------------------------------------------------------------------- likelihoods
# Gamma (Section 5, the MODIS application): y | mu ~ Gamma(shape alpha, rate alpha e^{-mu}),
# so E[y | mu] = e^mu; alpha is the auxiliary parameter xi of Section 2. With u = y e^{-mu}:
#   log p = alpha log alpha - log Gamma(alpha) + (alpha - 1) log y - alpha mu - alpha u,
#   d log p / d mu = alpha (u - 1),   W = alpha u  (> 0 for y > 0: log-concave in mu).
# Bernoulli and Poisson have no auxiliary parameter and ignore xi.
def log_lik(y: np.ndarray, mu: np.ndarray, lik: int, xi: float = 1.0) -> np.ndarray:
    if lik == LIK_BERNOULLI_LOGIT:
        # y mu - log(1 + e^mu)
        return y * mu - np.logaddexp(0.0, mu)
    if lik == LIK_GAMMA_LOG:
        a = float(xi)
        return a * np.log(a) - gammaln(a) + (a - 1.0) * np.log(y) - a * mu - a * y * np.exp(-mu)
    return y * mu - np.exp(mu) - gammaln(y + 1.0)


def grad_lik(y, mu, lik, xi: float = 1.0):
    if lik == LIK_BERNOULLI_LOGIT:
        return y - 1.0 / (1.0 + np.exp(-mu))
    if lik == LIK_GAMMA_LOG:
        return float(xi) * (y * np.exp(-mu) - 1.0)
    return y - np.exp(mu)


def W_lik(y, mu, lik, xi: float = 1.0):
    if lik == LIK_BERNOULLI_LOGIT:
        p = 1.0 / (1.0 + np.exp(-mu))
        return p * (1.0 - p)
    if lik == LIK_GAMMA_LOG:
        return float(xi) * y * np.exp(-mu)
    return np.exp(mu)


# ----------------------------------------------------------------------------- factor
@dataclasses.dataclass
class Factor:
    locs: np.ndarray      # Vecchia order
    order: np.ndarray     # order[k] = caller index of Vecchia row k
    N: np.ndarray
    A: np.ndarray
    D: np.ndarray
    B: sp.csr_matrix
    Sinv: sp.csr_matrix
    cov: int
    sigma2: float
    rho: float
    nugget: float

    @property
    def n(self):
        return len(self.D)


def knn_prev_fast(locs: np.ndarray, m: int) -> np.ndarray:
    """Exact N(i) for all rows for larger n: candidates from a k-d tree query
    (a library nearest-neighbour step), re-keyed with the exact (d2, j) key;
    rows whose candidate list cannot be proven complete fall back to brute force."""
    from scipy.spatial import cKDTree
    n = len(locs)
    if n <= 4096:
        return geometry.knn_prev(locs, m)
    K = min(n, 8 * m + 8)
    dist_t, cand = cKDTree(locs).query(locs, k=K)
    out = np.full((n, m), -1, np.int32)
    x, y = locs[:, 0], locs[:, 1]
    step = 20000
    for a in range(0, n, step):
        rows = np.arange(a, min(n, a + step))
        c = cand[rows]
        d2 = (x[rows, None] - x[c]) ** 2 + (y[rows, None] - y[c]) ** 2
        prev = c < rows[:, None]
        d2 = np.where(prev, d2, np.inf)
        o = np.lexsort((c, d2), axis=-1)
        cs = np.take_along_axis(c, o, -1)
        ds = np.take_along_axis(d2, o, -1)
        need = np.minimum(rows, m)
        kth = ds[np.arange(len(rows)), np.maximum(need - 1, 0)]
        bound = dist_t[rows, K - 1] ** 2 * (1.0 - 1e-12)
        ok = (need == 0) | ((kth < bound) & np.isfinite(kth)) | (K >= n)
        for r_i, i in enumerate(rows):
            k = need[r_i]
            if k == 0:
                continue
            if ok[r_i]:
                out[i, :k] = cs[r_i, :k]
            else:
                out[i] = geometry.knn_prev_rows(locs, m, [i])[0]
    return out


def build_factor(locs_user, order, cov, sigma2, rho, m, nugget, N=None) -> Factor:
    order = np.asarray(order, dtype=np.int64)
    locs = np.ascontiguousarray(locs_user[order])
    if N is None:
        N = geometry.knn_prev(locs, m) if len(locs) <= 4096 else knn_prev_fast(locs, m)
    A, D = vecchia.vecchia_factor(locs, N, cov, sigma2, rho, nugget)
    B = vecchia.B_matrix(N, A)
    return Factor(locs, order, N, A, D, B, vecchia.precision(B, D), cov, sigma2, rho, nugget)


def refit(f: Factor, sigma2, rho, nugget=None) -> Factor:
    nugget = 1e-10 * sigma2 if nugget is None else nugget
    A, D = vecchia.vecchia_factor(f.locs, f.N, f.cov, sigma2, rho, nugget)
    B = vecchia.B_matrix(f.N, A)
    return Factor(f.locs, f.order, f.N, A, D, B, vecchia.precision(B, D), f.cov, sigma2, rho, nugget)


def _lu(Amat: sp.spmatrix):
    return spla.splu(Amat.tocsc(), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                     options={"SymmetricMode": True})


def logdet_spd(Amat: sp.spmatrix) -> float:
    lu = _lu(Amat)
    return float(np.sum(np.log(np.abs(lu.U.diagonal()))) + np.sum(np.log(np.abs(lu.L.diagonal()))))


# ----------------------------------------------------------------------------- mode
@dataclasses.dataclass
class Mode:
    b: np.ndarray          # Vecchia order
    W: np.ndarray
    mu: np.ndarray
    y: np.ndarray
    F: np.ndarray
    lik: int
    iters: int
    psi: float
    xi: float = 1.0        # auxiliary likelihood parameter (gamma shape)


def psi(f: Factor, y, F, b, lik, xi: float = 1.0) -> float:
    return float(np.sum(log_lik(y, F + b, lik, xi)) - 0.5 * b @ (f.Sinv @ b))


def find_mode(f: Factor, y_user, F_user, lik, newton_tol=1e-9, max_iter=100, xi: float = 1.0) -> Mode:
    y = np.asarray(y_user, float)[f.order]
    F = np.zeros(f.n) if F_user is None else np.asarray(F_user, float)[f.order]
    b = np.zeros(f.n)
    ps = psi(f, y, F, b, lik, xi)
    it = 0
    for it in range(1, max_iter + 1):
        mu = F + b
        W = W_lik(y, mu, lik, xi)
        rhs = W * b + grad_lik(y, mu, lik, xi)
        b_new = _lu(sp.diags(W) + f.Sinv).solve(rhs)
        ps_new = psi(f, y, F, b_new, lik, xi)
        halvings = 0
        while ps_new < ps - 1e-12 * (1.0 + abs(ps)) and halvings < 30:
            b_new = b + 0.5 * (b_new - b)
            ps_new = psi(f, y, F, b_new, lik, xi)
            halvings += 1
        step = np.max(np.abs(b_new - b)) if f.n else 0.0
        b, ps = b_new, ps_new
        if step <= newton_tol * (1.0 + (np.max(np.abs(b)) if f.n else 0.0)):
            break
    mu = F + b
    return Mode(b=b, W=W_lik(y, mu, lik, xi), mu=mu, y=y, F=F, lik=lik, iters=it, psi=ps, xi=float(xi))


def mode_user(f: Factor, md: Mode) -> np.ndarray:
    out = np.empty(f.n)
    out[f.order] = md.b
    return out


# ----------------------------------------------------------------------------- L^VLA
def lml_parts(f: Factor, md: Mode) -> dict:
    nll = -float(np.sum(log_lik(md.y, md.mu, md.lik, md.xi)))
    quad = 0.5 * float(md.b @ (f.Sinv @ md.b))
    return {"neg_loglik": nll, "quad": quad, "sum_log_D": float(np.sum(np.log(f.D)))}


def lml_exact(f: Factor, md: Mode) -> tuple[float, float]:
    """(L^VLA, log det(Sigma_tilde W + I)) with the exact log-determinant."""
    p = lml_parts(f, md)
    ld = p["sum_log_D"] + logdet_spd(sp.diags(md.W) + f.Sinv)
    return p["neg_loglik"] + p["quad"] + 0.5 * ld, ld


def A_apply_fn(f: Factor, W):
    B, D = f.B, f.D
    return lambda v: W * v + B.T @ ((B @ v) / D)


def _tri_solvers(B: sp.csr_matrix):
    Bc = B.tocsc()
    lo = lambda v: spla.spsolve_triangular(B, v, lower=True)
    up = lambda v: spla.spsolve_triangular(Bc.T.tocsr(), v, lower=False)
    return lo, up


def precond_scale(f: Factor, W, prec: int) -> np.ndarray:
    """s with P^{-1/2} = diag(s) B^{-T}: VADU s = (W + 1/D)^{-1/2}, LVA s = D^{1/2}."""
    return 1.0 / np.sqrt(W + 1.0 / f.D) if prec == PREC_VADU else np.sqrt(f.D)


def logdet_P(f: Factor, W, prec: int) -> float:
    if prec == PREC_VADU:
        return float(np.sum(np.log(W + 1.0 / f.D)))
    return -float(np.sum(np.log(f.D)))


def slq_gammas(f: Factor, md: Mode, R: np.ndarray, prec: int = PREC_VADU, rtol=1e-14) -> np.ndarray:
    """gamma_i for each column of R (Rademacher, Vecchia row order)."""
    lo, up = _tri_solvers(f.B)
    s = precond_scale(f, md.W, prec)
    Aap = A_apply_fn(f, md.W)
    M = lambda v: s * up(Aap(lo(s * v)))   # P^{-1/2} A P^{-T/2} = S B^{-T} A B^{-1} S
    return np.array([krylov.lanczos_fr(M, R[:, j].copy(), rtol=rtol)[0] for j in range(R.shape[1])])


def probes(f: Factor, t: int, seed: int) -> np.ndarray:
    """Rademacher r (n x t) in Vecchia row order, drawn by caller point index."""
    return orng.rademacher(f.order, t, seed, orng.STREAM_PROBE)


def lml_slq(f: Factor, md: Mode, t: int, seed: int, prec: int = PREC_VADU, cols=None):
    """(L^VLA, logdet, gammas) with the same-probe SLQ estimate; ``cols`` selects a
    subset of the t probes (the estimate then averages over that subset)."""
    R = probes(f, t, seed)
    if cols is not None:
        R = R[:, cols]
    g = slq_gammas(f, md, R, prec)
    p = lml_parts(f, md)
    ld = p["sum_log_D"] + logdet_P(f, md.W, prec) + float(np.mean(g))
    return p["neg_loglik"] + p["quad"] + 0.5 * ld, ld, g


# ----------------------------------------------------------------------------- prediction
@dataclasses.dataclass
class PredFactor:
    Np: np.ndarray    # (n_p, m) Vecchia row indices of training neighbours
    Ap: np.ndarray    # (n_p, m)
    Dp: np.ndarray    # (n_p,)
    Bpo: sp.csr_matrix


def pred_factor(f: Factor, test_locs: np.ndarray, m: int) -> PredFactor:
    Np = geometry.knn_cross(f.locs, test_locs, m)
    n_p = len(test_locs)
    Ap = np.zeros((n_p, m))
    Dp = np.empty(n_p)
    k = min(m, f.n)
    sii = f.sigma2 + f.nugget
    if k == 0:
        Dp[:] = sii
    else:
        P = f.locs[Np[:, :k]]
        S_NN = vecchia.cov_fn(vecchia.dist(P[:, :, None, :], P[:, None, :, :]), f.cov, f.sigma2, f.rho)
        S_NN[:, np.arange(k), np.arange(k)] += f.nugget
        S_Ni = vecchia.cov_fn(vecchia.dist(P, test_locs[:, None, :]), f.cov, f.sigma2, f.rho)
        a = np.linalg.solve(S_NN, S_Ni[..., None])[..., 0]
        Ap[:, :k] = a
        Dp[:] = sii - (S_Ni * a).sum(1)
    rows = np.repeat(np.arange(n_p), m)
    cols = Np.ravel()
    ok = cols >= 0
    Bpo = sp.csr_matrix((-Ap.ravel()[ok], (rows[ok], cols[ok])), shape=(n_p, f.n))
    return PredFactor(Np, Ap, Dp, Bpo)


def pred_mean(pf: PredFactor, md: Mode, Fp) -> np.ndarray:
    return np.asarray(Fp, float) - pf.Bpo @ md.b


def pred_var_exact(f: Factor, md: Mode, pf: PredFactor, rows=None) -> np.ndarray:
    rows = np.arange(len(pf.Dp)) if rows is None else np.asarray(rows)
    if len(rows) == 0:
        return np.zeros(0)
    lu = _lu(sp.diags(md.W) + f.Sinv)
    Bt = pf.Bpo[rows].toarray().T                    # (n, r)
    X = lu.solve(Bt)
    return pf.Dp[rows] + np.sum(Bt * X, axis=0)


def pred_var_sim(f: Factor, md: Mode, pf: PredFactor, s: int, seed: int) -> np.ndarray:
    z1 = orng.gaussian(f.order, s, seed, orng.STREAM_SIM1)
    z2 = orng.gaussian(f.order, s, seed, orng.STREAM_SIM2)
    z3 = np.sqrt(md.W)[:, None] * z1 + f.B.T @ (z2 / np.sqrt(f.D)[:, None])
    U = _lu(sp.diags(md.W) + f.Sinv).solve(z3)
    z4 = pf.Bpo @ U
    return pf.Dp + np.mean(z4 * z4, axis=1)
