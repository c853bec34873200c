"""CUDA path vs the CPU oracle, through the C ABI, on the same seeded inputs.

Neighbour sets and level schedules must be bit-exact. The float64 path must
match the oracle within 1e-9 relative on the mode, L^VLA and predictive
variances; the factor within 1e-10 (D_i cancels digits and the oracle solves by LU, the kernel
by Cholesky). The mixed-precision path must reach
relative residual <= 1e-6 on every refined solve and 1e-4 relative on L^VLA.
"""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import geometry, krylov, laplace as la

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def vl():
    import paper_2310_12000_gb300 as vl
    vl.library()
    return vl


@pytest.fixture(scope="module")
def ctx(vl):
    return vl.Context(0, ws_bytes=4 << 30)


def _oracle_all(P, newton_tol=1e-10):
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=newton_tol)
    return f, md


FP64_TIGHT = dict(cg_tol=1e-12, newton_tol=1e-10, cg_max_iter=2000)


# ----------------------------------------------------------------------------- neighbours
def test_knn_golden_ties(ctx):
    g = json.load(open(os.path.join(GOLDEN, "knn_ties_m3.json")))
    N = ctx.knn_prev(np.array(g["locs"]), g["m"])
    assert N.tolist() == g["N"]


@pytest.mark.parametrize("case", ["uniform3000", "grid70", "uniform_m30", "tiny"])
def test_knn_prev_bitexact(ctx, case):
    rng = np.random.default_rng(11)
    if case == "uniform3000":
        locs, m = rng.random((3000, 2)), 10          # spans the brute-force head and the grid search
    elif case == "grid70":
        g = np.stack(np.meshgrid(np.arange(70), np.arange(70), indexing="ij"), -1).reshape(-1, 2) / 70.0
        locs, m = g[rng.permutation(len(g))], 10     # massive exact distance ties
    elif case == "uniform_m30":
        locs, m = rng.random((2500, 2)) * [3.0, 0.5], 30
    else:
        locs, m = rng.random((5, 2)), 8              # m > n
    N = ctx.knn_prev(locs, m)
    assert np.array_equal(N, geometry.knn_prev(locs, m))


def test_knn_prev_large_sampled(ctx):
    P = wl.make_problem("c2_n100k")
    locs = P.locs[P.order]
    N = ctx.knn_prev(locs, 20)
    rows = np.concatenate([np.arange(64), np.random.default_rng(0).choice(len(locs), 400, replace=False)])
    assert np.array_equal(N[rows], geometry.knn_prev_rows(locs, 20, rows))


def test_knn_cross_bitexact(ctx):
    rng = np.random.default_rng(5)
    tr = rng.random((4000, 2))
    te = np.concatenate([rng.random((300, 2)), tr[:20], [[-0.5, 0.5], [1.5, 1.5]]])
    for m in (1, 7, 20):
        assert np.array_equal(ctx.knn_cross(tr, te, m), geometry.knn_cross(tr, te, m))
    assert np.array_equal(ctx.knn_cross(tr[:3], te[:5], 6), geometry.knn_cross(tr[:3], te[:5], 6))


# ----------------------------------------------------------------------------- factor
@pytest.mark.parametrize("name,n", [("c1_n2000", None), ("c2_n100k", 5000)])
def test_factor_parity(ctx, vl, name, n):
    P = wl.make_problem(name, n=n)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    ex = fac.export()
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    assert np.array_equal(ex["N"], f.N)
    assert np.array_equal(ex["lev_fwd"], geometry.levels_forward(f.N))
    assert np.array_equal(ex["lev_bwd"], geometry.levels_backward(f.N))
    # D_i = Sigma_ii - w^T w cancels log10(Sigma_ii / D_i) digits, and the oracle solves
    # with LU while the kernel uses Cholesky: rounding alone separates them by up to
    # ~1e3 eps relative on the smallest D_i at this range; 1e-10 keeps 10x headroom.
    assert np.max(np.abs(ex["D"] - f.D) / f.D) < 1e-10
    assert np.max(np.abs(ex["A"] - f.A)) < 1e-10 * max(1.0, np.max(np.abs(f.A)))
    info = fac.info()
    assert info["nlev_fwd"] == geometry.levels_forward(f.N).max() + 1


def test_factor_edge_cases(ctx):
    for n, m in [(1, 5), (2, 1), (7, 0), (30, 29), (40, 64)]:
        P = wl.tiny_problem(n, m)
        fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, m)
        ex = fac.export()
        f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, m, P.nugget)
        assert np.array_equal(ex["N"], f.N)
        assert np.allclose(ex["D"], f.D, rtol=1e-11, atol=0)
        assert np.allclose(ex["A"], f.A, rtol=1e-9, atol=1e-11)


def test_refit_matches_fresh_build(ctx):
    P = wl.make_problem("c1_n2000", n=800)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    fac.refit(1.7, 0.23)
    f = la.refit(la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget), 1.7, 0.23)
    ex = fac.export()
    assert np.max(np.abs(ex["D"] - f.D) / f.D) < 1e-12


# ----------------------------------------------------------------------------- operators
@pytest.mark.parametrize("t", [1, 5, 40])
def test_operator_parity(ctx, vl, t):
    P = wl.make_problem("c1_n2000", n=700)
    f, md = _oracle_all(P)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    st = fac.find_mode(P.lik, P.y, P.F, vl.Opts.make(**FP64_TIGHT))
    X = np.random.default_rng(t).standard_normal((P.n, t))
    Xv = X[f.order]
    B, D, W = f.B, f.D, md.W
    Bd = B.toarray()
    ref = {
        vl.OP_B: B @ Xv,
        vl.OP_BT: B.T @ Xv,
        vl.OP_A: W[:, None] * Xv + B.T @ ((B @ Xv) / D[:, None]),
        vl.OP_BINV: np.linalg.solve(Bd, Xv),
        vl.OP_BTINV: np.linalg.solve(Bd.T, Xv),
        vl.OP_SIGMA: np.linalg.solve(Bd, D[:, None] * np.linalg.solve(Bd.T, Xv)),
    }
    ref[vl.OP_PINV] = np.linalg.solve(Bd, np.linalg.solve(Bd.T, Xv) / (W + 1 / D)[:, None])
    ref[vl.OP_A2] = ref[vl.OP_SIGMA] + Xv / W[:, None]
    for op, Yv in ref.items():
        Y = st.apply(op, X)
        Yu = np.empty_like(Yv)
        Yu[f.order] = Yv
        err = np.max(np.abs(Y - Yu)) / np.max(np.abs(Yu))
        assert err < 1e-9, (op, err)


def test_pcg_T_matches_oracle_pcg(ctx, vl):
    P = wl.make_problem("c1_n2000", n=900)
    f, md = _oracle_all(P)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    st = fac.find_mode(P.lik, P.y, P.F, vl.Opts.make(**FP64_TIGHT))
    R = np.random.default_rng(3).standard_normal((P.n, 3))
    U, Td, To, it, rel = st.pcg_solve(R, vl.Opts.make(cg_tol=1e-10, cg_max_iter=500), lmax=500)
    Aop = la.A_apply_fn(f, md.W)
    Pm = la.precond_scale(f, md.W, la.PREC_VADU) ** 2
    lo, up = la._tri_solvers(f.B)
    Pinv = lambda v: lo(Pm * up(v))
    for j in range(3):
        u, dT, oT, nit, rl, _ = krylov.pcg_with_T(Aop, Pinv, R[f.order, j], 1e-10, 500)
        # two float64 CG runs agree on the leading T entries; late entries separate
        # by rounding once Ritz values converge (loss of orthogonality), so only the
        # first 12 are compared entrywise and the iteration counts within 2.
        assert abs(int(it[j]) - nit) <= 2
        k = min(12, nit)
        assert np.allclose(Td[j, :k], dT[:k], rtol=1e-9)
        assert np.allclose(To[j, :k - 1], oT[:k - 1], rtol=1e-9)
        uu = np.empty_like(u)
        uu[f.order] = u
        assert np.max(np.abs(U[:, j] - uu)) < 1e-8 * np.max(np.abs(uu))
        assert rel[j] <= 1e-10


# ----------------------------------------------------------------------------- Laplace
@pytest.mark.parametrize("name,n", [("c1_n2000", None), ("c3_grid1m", 3000)])
def test_mode_and_lml_parity_fp64(ctx, vl, name, n):
    P = wl.make_problem(name, n=n)
    t = 50
    opts = vl.Opts.make(t=t, **FP64_TIGHT)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts)
    st = fac.find_mode(P.lik, P.y, P.F, opts)
    lml, stats = st.log_marglik(opts, with_stats=True)
    f, md = _oracle_all(P)
    b_ref = la.mode_user(f, md)
    assert np.max(np.abs(st.mode - b_ref)) / np.max(np.abs(b_ref)) < 1e-9
    L_ref, ld_ref, g_ref = la.lml_slq(f, md, t, 1)
    g = st.slq_gammas(t)
    assert np.max(np.abs(g - g_ref) / np.maximum(np.abs(g_ref), 1.0)) < 1e-9
    assert abs(lml - L_ref) / abs(L_ref) < 1e-9
    # and the estimate is statistically consistent with the exact Laplace value
    L_ex, _ = la.lml_exact(f, md)
    assert abs(lml - L_ex) < 4 * 0.5 * stats["slq_stderr"] + 1e-9 * abs(L_ex)


def test_lva_preconditioner_parity(ctx, vl):
    P = wl.make_problem("c1_n2000", n=1000)
    opts = vl.Opts.make(t=20, precond=vl.PREC_LVA, **FP64_TIGHT)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts)
    st = fac.find_mode(P.lik, P.y, P.F, opts)
    lml = st.log_marglik(opts)
    f, md = _oracle_all(P)
    L_ref, _, g_ref = la.lml_slq(f, md, 20, 1, prec=la.PREC_LVA)
    assert abs(lml - L_ref) / abs(L_ref) < 1e-9


def test_pred_parity_fp64(ctx, vl):
    P = wl.make_problem("c1_n2000")
    opts = vl.Opts.make(s=100, **FP64_TIGHT)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts)
    st = fac.find_mode(P.lik, P.y, P.F, opts)
    mean, var = st.pred_var(P.test_locs, P.Fp, opts)
    f, md = _oracle_all(P)
    pf = la.pred_factor(f, P.test_locs, P.m)
    assert np.max(np.abs(mean - la.pred_mean(pf, md, P.Fp))) < 1e-9 * (1 + np.max(np.abs(mean)))
    v_ref = la.pred_var_sim(f, md, pf, 100, 1)
    assert np.max(np.abs(var - v_ref) / v_ref) < 1e-9


def test_mixed_precision_lml_and_residuals(ctx, vl):
    P = wl.make_problem("c1_n2000")
    o64 = vl.Opts.make(t=50, **FP64_TIGHT)
    o32 = vl.Opts.make(t=50, precision=vl.FP32_REFINE, cg_tol=1e-6, newton_tol=1e-7)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, o64)
    st32 = fac.find_mode(P.lik, P.y, P.F, o32)
    lml32, s32 = st32.log_marglik(o32, with_stats=True)
    f, md = _oracle_all(P)
    L_ref, _, _ = la.lml_slq(f, md, 50, 1)
    assert abs(lml32 - L_ref) / abs(L_ref) < 1e-4
    b_ref = la.mode_user(f, md)
    assert np.max(np.abs(st32.mode - b_ref)) / np.max(np.abs(b_ref)) < 1e-4
    mean, var = st32.pred_var(P.test_locs, P.Fp, vl.Opts.make(s=64, precision=vl.FP32_REFINE, cg_tol=1e-6))
    pf = la.pred_factor(f, P.test_locs, P.m)
    v_ref = la.pred_var_sim(f, md, pf, 64, 1)
    assert np.max(np.abs(var - v_ref) / v_ref) < 1e-4


def test_poisson_offset_and_full_conditioning(ctx, vl):
    P = wl.tiny_problem(60, 59, lik=wl.LIK_POISSON_LOG, rho=0.3, F0=0.5, n_test=9)
    opts = vl.Opts.make(t=8, s=16, **FP64_TIGHT)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts)
    st = fac.find_mode(P.lik, P.y, P.F, opts)
    lml = st.log_marglik(opts)
    f, md = _oracle_all(P)
    assert np.max(np.abs(st.mode - la.mode_user(f, md))) < 1e-9 * (1 + np.max(np.abs(st.mode)))
    L_ref, _, _ = la.lml_slq(f, md, 8, 1)
    assert abs(lml - L_ref) / abs(L_ref) < 1e-9
