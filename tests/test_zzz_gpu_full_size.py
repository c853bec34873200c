"""The benchmark's timed step at full size (the n = 1e6 grid-with-gaps workload, Poisson,
Matern-1.5, m = 20; float32 Krylov with float64 refinement, VADU, t = 50), checked by the
oracle where it can work at that size (tests/fullsize.py): neighbour sets and factor rows of
sampled rows, the level recurrences on every row, the stationarity of the mode, the assembly
of L^VLA from its parts and Theorem 3.1's bound on every SLQ term. The slowest GPU test, so
it runs last.

Tolerances. The factor rows: LU and Cholesky, both correct in float64, differ here by up to
3e-12 on A and 1e-11 relative on D (condition numbers of Sigma_N up to 6e5); 1e-9 keeps 100x
headroom. Stationarity: the final Newton iterate is the output of a refined solve stopped at
||rhs - A x|| <= cg_tol ||rhs||, and its residual equals grad psi up to O(step^2), so
||grad psi|| <= 10 cg_tol ||rhs||. The L^VLA assembly sums the same float64 terms in another
order: 1e-9 relative."""
import numpy as np
import pytest

import fullsize as fs
import workloads as wl
from oracle import laplace as la

pytestmark = pytest.mark.gpu


def test_bench_step_at_full_size():
    import torch

    import paper_2310_12000_gb300 as vl
    vl.library()
    P = wl.make_problem("c3_grid1m", seed=1)
    n, m, t, cg_tol = P.n, P.m, 50, 1e-6
    ctx = vl.Context(0, ws_bytes=24 << 30)
    opts = vl.Opts.make(precision=vl.FP32_REFINE, t=t, cg_tol=cg_tol, newton_tol=1e-7, cg_max_iter=3000,
                        precond=vl.PREC_VADU)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, m, opts)
    y_d = torch.from_numpy(P.y).to("cuda:0")
    F_d = torch.from_numpy(P.F).to("cuda:0")
    mode_d = torch.empty(n, dtype=torch.float64, device="cuda:0")
    fac.refit(P.sigma2, P.rho, opts)
    st = fac.find_mode(P.lik, y_d, F_d, opts, mode_out=mode_d)
    lml, stats = st.log_marglik(opts, with_stats=True)
    gam = st.slq_gammas(t)
    mstats = st.mode_stats()
    torch.cuda.synchronize()
    mode = mode_d.cpu().numpy()
    ex = fac.export()
    info = fac.info()
    st.close()
    fac.close()
    ctx.close()

    order = P.order
    locs_v = P.locs[order]
    # neighbours bit-exact and factor rows on sampled rows
    rows = fs.sample_rows(n, m, 200, 0)
    N_ref, A_ref, D_ref = fs.factor_rows(locs_v, rows, m, P.cov, P.sigma2, P.rho, P.nugget)
    assert np.array_equal(ex["N"][rows], N_ref)
    assert np.max(np.abs(ex["A"][rows] - A_ref)) < 1e-9 * max(1.0, np.max(np.abs(A_ref)))
    assert np.max(np.abs(ex["D"][rows] - D_ref) / D_ref) < 1e-9
    # level schedules: the recurrences on every row
    assert fs.level_recurrences_hold(ex["N"], ex["lev_fwd"], ex["lev_bwd"]) == (True, True)
    assert info["nlev_fwd"] == int(ex["lev_fwd"].max()) + 1
    assert info["nlev_bwd"] == int(ex["lev_bwd"].max()) + 1
    # the mode is stationary to the refinement tolerance
    y_v, F_v, b_v = P.y[order], P.F[order], mode[order]
    assert np.all(np.isfinite(b_v))
    g, r = fs.stationarity(ex["N"], ex["A"], ex["D"], y_v, F_v, b_v, P.lik)
    assert g <= 10 * cg_tol * r, (g, r)
    assert mstats["true_relres_max"] <= cg_tol and mstats["newton_iters"] >= 1
    # L^VLA assembled from the factor, the mode and the SLQ terms
    assert np.all(np.isfinite(gam)) and abs(gam.mean() - stats["slq_mean"]) <= 1e-12 * max(1.0, abs(gam.mean()))
    L_cpu, ld_cpu = fs.lml_from_parts(ex["N"], ex["A"], ex["D"], y_v, F_v, b_v, P.lik, gam.mean())
    assert abs(lml - L_cpu) <= 1e-9 * abs(L_cpu), (lml, L_cpu)
    assert abs(stats["logdet"] - ld_cpu) <= 1e-9 * max(abs(ld_cpu), 1.0)
    # Theorem 3.1: every SLQ term is at least n log min_i (D_i W_ii + 1)^{-1}
    W = la.W_lik(y_v, F_v + b_v, P.lik)
    assert np.all(gam / n >= fs.gamma_lower_bound(ex["D"], W))
