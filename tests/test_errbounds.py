"""The rounding-error bounds of tests/errbounds.py on CPU: results computed in float32 by plain
row loops (one dot product per row, in the working precision) stay inside them, and a result
moved a few bounds away from the exact one is caught."""
import numpy as np

import errbounds as eb
import workloads as wl
from oracle import laplace as la


def _f32_product(B, X, transpose=False):
    M = (B.T if transpose else B).tocsr().astype(np.float32)
    X32 = X.astype(np.float32)
    Y = np.empty_like(X32)
    for i in range(M.shape[0]):
        a, b = M.indptr[i], M.indptr[i + 1]
        Y[i] = (M.data[a:b, None] * X32[M.indices[a:b]]).sum(0, dtype=np.float32)
    return Y.astype(np.float64)


def _f32_solve(B, X, transpose=False):
    """Substitution in float32: y_i = x_i - sum_{j<i} B_ij y_j (forward, B lower), or the
    backward recurrence for B^T, each row one float32 dot product."""
    M = (B.T if transpose else B).tocsr().astype(np.float32)
    X32 = X.astype(np.float32)
    n = M.shape[0]
    Y = np.zeros_like(X32)
    rows = range(n - 1, -1, -1) if transpose else range(n)
    for i in rows:
        a, b = M.indptr[i], M.indptr[i + 1]
        idx, val = M.indices[a:b], M.data[a:b]
        keep = idx != i
        acc = X32[i] - (val[keep, None] * Y[idx[keep]]).sum(0, dtype=np.float32)
        Y[i] = acc.astype(np.float32)
    return Y.astype(np.float64)


def test_float32_results_lie_inside_the_bounds_and_planted_errors_do_not():
    P = wl.make_problem("c1_n2000", n=300)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    B = f.B
    X = np.random.default_rng(4).standard_normal((P.n, 3))
    Bd = B.toarray()
    aB, off = eb.abs_parts(B)
    kf, kb = eb.row_terms(off), eb.row_terms(off.T.tocsr())
    aBinv = np.abs(np.linalg.inv(Bd))
    cases = {
        "B": (_f32_product(B, X), Bd @ X, eb.product_bound(aB, X, kf, eb.U32)),
        "BT": (_f32_product(B, X, True), Bd.T @ X, eb.product_bound(aB.T.tocsr(), X, kb, eb.U32)),
    }
    Yf = _f32_solve(B, X)
    cases["BINV"] = (Yf, np.linalg.solve(Bd, X), eb.solve_bound(aBinv, off, X, Yf, kf, eb.U32))
    Yb = _f32_solve(B, X, True)
    cases["BTINV"] = (Yb, np.linalg.solve(Bd.T, X),
                      eb.solve_bound(aBinv.T, off.T.tocsr(), X, Yb, kb, eb.U32))
    for name, (got, ref, bound) in cases.items():
        err = np.abs(got - ref)
        assert np.all(err <= eb.BOUND_SLACK * bound), name
        # the float32 rounding is visible (the check is not vacuous) ...
        assert err.max() > 1e-3 * bound.max(), name
        # ... and an error of a few bounds in one entry is caught
        bad = got.copy()
        k = np.unravel_index(np.argmax(bound), bound.shape)
        bad[k] += 3 * eb.BOUND_SLACK * bound[k]
        assert not np.all(np.abs(bad - ref) <= eb.BOUND_SLACK * bound), name
    # the float64 bounds are ~2^29 times tighter
    assert eb.gamma(kf, eb.U64) < 1e-8 * eb.gamma(kf, eb.U32)


def test_backward_recurrence_rows_have_more_terms_than_m():
    """Rows of B^T list every row that uses a point as a neighbour: more than m + 1 terms, so
    the bound of the backward solves must count them."""
    P = wl.make_problem("c1_n2000", n=300)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    _, off = eb.abs_parts(f.B)
    assert eb.row_terms(off) == P.m + 1
    assert eb.row_terms(off.T.tocsr()) > P.m + 1
