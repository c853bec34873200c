"""The full-size checks (tests/fullsize.py) on CPU: at a size where the oracle computes
everything, each check accepts the oracle's own outputs and rejects a planted mistake, so
that the GPU test at n = 1e6 relies on checks that are known to work."""
import numpy as np

import fullsize as fs
import workloads as wl
from oracle import geometry, laplace as la


def _oracle_run():
    P = wl.make_problem("c3_grid1m", n=3000)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-12)
    L, ld, gam = la.lml_slq(f, md, 12, 1)
    return P, f, md, L, ld, gam


def test_checks_accept_the_oracle_and_reject_planted_mistakes():
    P, f, md, L, ld, gam = _oracle_run()
    locs_v = P.locs[P.order]
    rows = fs.sample_rows(P.n, P.m, 60, 0)
    assert rows[0] == 0 and rows[-1] == P.n - 1
    N, A, D = fs.factor_rows(locs_v, rows, P.m, P.cov, P.sigma2, P.rho, P.nugget)
    assert np.array_equal(N, f.N[rows])
    assert np.max(np.abs(A - f.A[rows])) < 1e-12 and np.max(np.abs(D - f.D[rows]) / f.D[rows]) < 1e-12
    # a neighbour list of another row is not accepted
    assert not np.array_equal(N[5:], f.N[rows[5:] - 1])

    lf, lb = geometry.levels_forward(f.N), geometry.levels_backward(f.N)
    assert fs.level_recurrences_hold(f.N, lf, lb) == (True, True)
    bad = lf.copy()
    bad[np.argmax(lf)] += 1
    assert fs.level_recurrences_hold(f.N, bad, lb)[0] is False
    bad = lb.copy()
    bad[np.nonzero(lb == 0)[0][0]] = 1
    assert fs.level_recurrences_hold(f.N, lf, bad)[1] is False
    bad = lf.copy()
    bad[np.nonzero(lf > 1)[0][0]] -= 1
    assert fs.level_recurrences_hold(f.N, bad, lb)[0] is False

    y_v, F_v = P.y[P.order], P.F[P.order]
    g, r = fs.stationarity(f.N, f.A, f.D, y_v, F_v, md.b, P.lik)
    assert g <= 1e-9 * r
    g2, r2 = fs.stationarity(f.N, f.A, f.D, y_v, F_v, md.b * (1 + 1e-4), P.lik)
    assert g2 > 1e-5 * r2

    L2, ld2 = fs.lml_from_parts(f.N, f.A, f.D, y_v, F_v, md.b, P.lik, gam.mean())
    assert abs(L2 - L) < 1e-12 * abs(L) and abs(ld2 - ld) < 1e-12 * abs(ld)
    L3, _ = fs.lml_from_parts(f.N, f.A, f.D, y_v, F_v, md.b, P.lik, gam.mean() + 1e-3 * abs(gam.mean()))
    assert abs(L3 - L) > 1e-9 * abs(L)

    lb_g = fs.gamma_lower_bound(f.D, md.W)
    assert np.all(gam / P.n >= lb_g)


def test_solve_backward_error_accepts_exact_solves_and_rejects_planted_mistakes():
    import scipy.sparse.linalg as spla
    P = wl.make_problem("c3_grid1m", n=3000)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    X = np.random.default_rng(2).standard_normal((P.n, 4))
    kf, kb = fs.max_row_terms(f.N), fs.max_row_terms(f.N, transpose=True)
    assert kf == P.m + 1 and kb > kf
    u = 2.0 ** -53
    Y = spla.spsolve_triangular(f.B.tocsr(), X, lower=True)
    assert fs.solve_backward_error(f.N, f.A, X, Y) <= kf * u * 4
    Yt = spla.spsolve_triangular(f.B.T.tocsr(), X, lower=False)
    assert fs.solve_backward_error(f.N, f.A, X, Yt, transpose=True) <= kb * u * 4
    # one wrong entry, a transposed solve and a solve with another row's weights are caught
    bad = Y.copy()
    bad[1234, 2] *= 1 + 1e-9
    assert fs.solve_backward_error(f.N, f.A, X, bad) > 1e3 * kf * u
    assert fs.solve_backward_error(f.N, f.A, X, Yt) > 1e3 * kf * u
    A2 = f.A.copy()
    A2[[10, 11]] = A2[[11, 10]]
    assert fs.solve_backward_error(f.N, A2, X, Y) > 1e3 * kf * u
