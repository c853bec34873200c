"""Every form of the level-scheduled triangular solves against the oracle, through the C ABI.

The preconditioners of Section 3.1.1 and Sigma_tilde = B^{-1} D B^{-T} are applied by solves
with B and B^T. A solve runs in one of three forms: one block with x in shared memory
(single-column solves of small systems), one thread-block cluster, or the cooperative grid
with a bounded software barrier per level (large problems; its narrow leading and trailing
levels run in one block, the leading ones of single-column forward solves with x in shared
memory). The automatic choice depends on n, t and the widest level, so the small parity cases
elsewhere reach only the first two; here each form is forced (vl_ctx_set_solve_form; "grid_all"
puts every level on the grid barrier) and checked:

* every operator of vl_apply at t = 1, 5, 40 and 50, in float64 and float32, element by
  element against dense float64 algebra on the library's own factor under the rounding-error
  bound of the operator (tests/errbounds.py: gamma_k of the rows' dot products, propagated
  through |B^{-1}| for the solves), and float64 results within 1e-9 of the oracle's operator;
* the Laplace mode, L^VLA, every SLQ term (float64, 1e-9) and the mixed-precision L^VLA
  (1e-4) with the whole path in that form;
* at n = 300,000 of the grid workload: neighbour sets and factor rows of sampled rows against
  the oracle, and the componentwise backward error of B^{-1} X and B^{-T} X on every element
  (Higham, Thm 8.5: below gamma_k, rows of at most k terms);
* a tuned and an untuned context give bit-identical solves.
"""
import numpy as np
import pytest

import scipy.linalg as sla

import errbounds as eb
import fullsize as fs
import workloads as wl
from oracle import laplace as la, vecchia

pytestmark = pytest.mark.gpu

FORMS = ["shared", "cluster", "grid", "grid_all", "tile"]
FP64_TIGHT = dict(cg_tol=1e-12, newton_tol=1e-10, cg_max_iter=2000)


@pytest.fixture(scope="module")
def vl():
    import paper_2310_12000_gb300 as vl
    vl.library()
    return vl


@pytest.fixture(scope="module")
def ctx(vl):
    c = vl.Context(0, ws_bytes=8 << 30)
    yield c
    c.set_solve_form(vl.SOLVE_AUTO)


def _form(vl, name):
    return {"auto": vl.SOLVE_AUTO, "shared": vl.SOLVE_SHARED, "cluster": vl.SOLVE_CLUSTER,
            "grid": vl.SOLVE_GRID, "grid_all": vl.SOLVE_GRID_ALL, "tile": vl.SOLVE_TILE}[name]


_CACHE = {}


def _oracle(P, key):
    if key not in _CACHE:
        f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
        md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-10)
        _CACHE[key] = (f, md)
    return _CACHE[key]


@pytest.fixture(scope="module")
def op_case(ctx, vl):
    """A factor and a mode (float64, automatic forms) of the c1 recipe at n = 700; the
    operators are then applied with each forced form. The rounding-error bounds are taken
    around the operator the library holds (its exported B and D, and W at its own mode),
    since the oracle's B, D and mode differ from those by more than a rounding (LU against
    Cholesky, Newton's stopping rule); the factor and the mode are compared with the oracle
    by the parity tests, and here every result also within 1e-9 of the oracle's operator."""
    P = wl.make_problem("c1_n2000", n=700)
    f, md = _oracle(P, "c1_700")
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    ctx.set_solve_form(vl.SOLVE_AUTO)
    st = fac.find_mode(P.lik, P.y, P.F, vl.Opts.make(**FP64_TIGHT))
    ex = fac.export()
    y_v, F_v = P.y[f.order], P.F[f.order]
    W = la.W_lik(y_v, F_v + st.mode[f.order], P.lik)
    lib = dict(B=vecchia.B_matrix(ex["N"], ex["A"]), D=ex["D"], W=W)
    return P, f, md, st, lib


def _refs(vl, B, D, W, Xv):
    """Every operator of vl_apply by dense float64 algebra (triangular substitutions)."""
    Bd = B.toarray()
    dsc = 1.0 / (W + 1.0 / D)
    ref = {vl.OP_B: Bd @ Xv, vl.OP_BT: Bd.T @ Xv,
           vl.OP_A: W[:, None] * Xv + Bd.T @ ((Bd @ Xv) / D[:, None]),
           vl.OP_BINV: sla.solve_triangular(Bd, Xv, lower=True, unit_diagonal=True),
           vl.OP_BTINV: sla.solve_triangular(Bd.T, Xv, lower=False, unit_diagonal=True)}
    ref[vl.OP_SIGMA] = sla.solve_triangular(Bd, D[:, None] * ref[vl.OP_BTINV], lower=True, unit_diagonal=True)
    ref[vl.OP_PINV] = sla.solve_triangular(Bd, dsc[:, None] * ref[vl.OP_BTINV], lower=True, unit_diagonal=True)
    ref[vl.OP_A2] = ref[vl.OP_SIGMA] + Xv / W[:, None]
    return ref, dsc


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("t", [1, 5, 40, 50])
@pytest.mark.parametrize("form", FORMS)
def test_operators_by_form(ctx, vl, op_case, form, t, prec):
    P, f, md, st, lib = op_case
    ops = {"A": vl.OP_A, "PINV": vl.OP_PINV, "B": vl.OP_B, "BT": vl.OP_BT, "BINV": vl.OP_BINV,
           "BTINV": vl.OP_BTINV, "SIGMA": vl.OP_SIGMA, "A2": vl.OP_A2}
    opts = vl.Opts.make(precision=vl.FP64 if prec == "fp64" else vl.FP32_REFINE)
    X = np.random.default_rng(100 + t).standard_normal((P.n, t))
    Xv = X[f.order]
    ctx.set_solve_form(_form(vl, form))
    try:
        Y = {op: st.apply(op, X, opts)[f.order] for op in ops.values()}
    finally:
        ctx.set_solve_form(vl.SOLVE_AUTO)
    # around the library's own operator: its rounding error bound (float64 results also carry
    # the float64 reference's own rounding, of the same bound)
    ref, dsc = _refs(vl, lib["B"], lib["D"], lib["W"], Xv)
    u = eb.U64 if prec == "fp64" else eb.U32
    bound = eb.operator_bounds(lib["B"], lib["D"], lib["W"], dsc, Xv, Y, ops, u)
    both = 2.0 if prec == "fp64" else 1.0
    for name, op in ops.items():
        err = np.abs(Y[op] - ref[op])
        ok = err <= eb.BOUND_SLACK * both * bound[op]
        assert ok.all(), (form, t, prec, name, float((err / bound[op]).max()))
    # against the oracle's operator (its factor, its mode)
    if prec == "fp64":
        oref, _ = _refs(vl, f.B, f.D, md.W, Xv)
        for name, op in ops.items():
            err = np.abs(Y[op] - oref[op]).max()
            assert err <= 1e-9 * np.abs(oref[op]).max(), (form, t, name, err)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name,n", [("c1_n2000", None), ("c3_grid1m", 3000)])
def test_mode_and_lml_by_form(ctx, vl, form, name, n):
    P = wl.make_problem(name, n=n)
    t = 50
    opts = vl.Opts.make(t=t, **FP64_TIGHT)
    f, md = _oracle(P, (name, n))
    ctx.set_solve_form(_form(vl, form))
    try:
        fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts)
        st = fac.find_mode(P.lik, P.y, P.F, opts)
        lml = st.log_marglik(opts)
        g = st.slq_gammas(t)
        o32 = vl.Opts.make(t=t, precision=vl.FP32_REFINE, cg_tol=1e-6, newton_tol=1e-7)
        st32 = fac.find_mode(P.lik, P.y, P.F, o32)
        lml32, s32 = st32.log_marglik(o32, with_stats=True)
    finally:
        ctx.set_solve_form(vl.SOLVE_AUTO)
    b_ref = la.mode_user(f, md)
    assert np.max(np.abs(st.mode - b_ref)) / np.max(np.abs(b_ref)) < 1e-9
    L_ref, _, g_ref = la.lml_slq(f, md, t, 1)
    assert np.max(np.abs(g - g_ref) / np.maximum(np.abs(g_ref), 1.0)) < 1e-9
    assert abs(lml - L_ref) / abs(L_ref) < 1e-9
    assert abs(lml32 - L_ref) / abs(L_ref) < 1e-4
    assert st32.mode_stats()["true_relres_max"] <= 1e-6


def test_forced_form_that_cannot_run_is_refused(ctx, vl, op_case):
    """A forced shared-memory solve of a system too large for one block's shared memory
    fails cleanly, and the context keeps working."""
    P = wl.make_problem("c1_n2000", n=30000)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    st = fac.find_mode(P.lik, P.y, P.F, vl.Opts.make(cg_tol=1e-8))
    ctx.set_solve_form(vl.SOLVE_SHARED)
    try:
        with pytest.raises(vl.VLError) as e:
            st.apply(vl.OP_BINV, np.ones((P.n, 1)), vl.Opts.make())
        assert e.value.status == 1 and "SHARED" in str(e.value)
    finally:
        ctx.set_solve_form(vl.SOLVE_AUTO)
    with pytest.raises(vl.VLError):
        ctx.set_solve_form(7)
    Y = st.apply(vl.OP_B, np.ones((P.n, 1)), vl.Opts.make())
    assert np.all(np.isfinite(Y))


@pytest.mark.parametrize("form", ["auto", "grid", "grid_all", "cluster", "tile"])
def test_large_solves_by_form(ctx, vl, form):
    """n = 300,000 of the grid-with-gaps workload (m = 20, hundreds of levels)."""
    P = wl.make_problem("c3_grid1m", n=300_000)
    n, m = P.n, P.m
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, m)
    ex = fac.export()
    locs_v = P.locs[P.order]
    rows = fs.sample_rows(n, m, 120, 1)
    N_ref, A_ref, D_ref = fs.factor_rows(locs_v, rows, m, P.cov, P.sigma2, P.rho, P.nugget)
    assert np.array_equal(ex["N"][rows], N_ref)
    assert np.max(np.abs(ex["A"][rows] - A_ref)) < 1e-9 * max(1.0, np.max(np.abs(A_ref)))
    assert np.max(np.abs(ex["D"][rows] - D_ref) / D_ref) < 1e-9
    st = fac.find_mode(P.lik, P.y, P.F, vl.Opts.make(precision=vl.FP32_REFINE, cg_tol=1e-6, newton_tol=1e-6,
                                                      cg_max_iter=3000))
    kf, kb = fs.max_row_terms(ex["N"]), fs.max_row_terms(ex["N"], transpose=True)
    ctx.set_solve_form(_form(vl, form))
    try:
        for prec, u in (("fp64", eb.U64), ("fp32", eb.U32)):
            opts = vl.Opts.make(precision=vl.FP64 if prec == "fp64" else vl.FP32_REFINE)
            for t in (1, 50):
                X = np.random.default_rng(t).standard_normal((n, t))
                Xv = X[P.order]
                Y = st.apply(vl.OP_BINV, X, opts)[P.order]
                Yt = st.apply(vl.OP_BTINV, X, opts)[P.order]
                assert np.all(np.isfinite(Y)) and np.all(np.isfinite(Yt))
                # X and the weights are rounded to the working precision first: 2u more
                w = fs.solve_backward_error(ex["N"], ex["A"], Xv, Y)
                wt = fs.solve_backward_error(ex["N"], ex["A"], Xv, Yt, transpose=True)
                assert w <= eb.BOUND_SLACK * (eb.gamma(kf, u) + 2 * u), (prec, t, w)
                assert wt <= eb.BOUND_SLACK * (eb.gamma(kb, u) + 2 * u), (prec, t, wt)
    finally:
        ctx.set_solve_form(vl.SOLVE_AUTO)


def test_tuned_launches_give_identical_results(vl):
    """The launch tuner only picks among parameters that change no result (blocks per SM,
    dependency rows in flight, thread-block clusters): a tuned context and an untuned one give
    bit-identical solves, in the call that tunes (every candidate launched in turn, the last
    one's result kept) and after the choice is cached."""
    P = wl.make_problem("c3_grid1m", n=300_000)
    outs = []
    for tune in (True, False):
        c = vl.Context(0, ws_bytes=4 << 30)
        c.set_autotune(tune)
        fac = c.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
        st = fac.find_mode(P.lik, P.y, P.F, vl.Opts.make(precision=vl.FP32_REFINE, cg_tol=1e-6, newton_tol=1e-6,
                                                          cg_max_iter=3000))
        if tune:
            vl.tune_reset()            # the first solve of each kind below tunes again
        res = []
        for t in (1, 50):
            X = np.random.default_rng(t).standard_normal((P.n, t))
            o = vl.Opts.make(precision=vl.FP32_REFINE)
            for _ in range(2):
                res.append(st.apply(vl.OP_BINV, X, o))
                res.append(st.apply(vl.OP_BTINV, X, o))
        outs.append(res)
        c.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    rep = vl.tune_report()
    assert rep and all(len(r["ms"]) >= 2 and 0 <= r["choice"] < len(r["ms"]) for r in rep)
