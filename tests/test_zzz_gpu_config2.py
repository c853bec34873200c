"""The uniform n = 1e5 workload at its full size (Matern-1.5, range 0.05, m = 20, Bernoulli-logit,
t = 50 probes, PCG tolerance 1e-6, predictive means and variances at 1e4 test points from s = 100
simulation vectors), on the float64 path and the float32 path with float64 refinement. At this
size the oracle works row by row, not globally, so the test checks: neighbour sets bit-exact and
factor rows within 1e-9 of the oracle's on sampled rows; the mixed path against the float64 path
within the stated 1e-4 on the mode, L^VLA and the predictive mean and variance (the same probes
and simulation vectors on both); every refined float64 residual (Newton and SLQ probe solves)
at or below 1e-6; and the SLQ standard error small against L^VLA."""
import numpy as np
import pytest

import fullsize as fs
import workloads as wl

pytestmark = pytest.mark.gpu


def test_uniform_n100k_fp64_and_mixed():
    import paper_2310_12000_gb300 as vl
    vl.library()
    P = wl.make_problem("c2_n100k")
    n, m = P.n, P.m
    ctx = vl.Context(0, ws_bytes=16 << 30)
    o64 = vl.Opts.make(precision=vl.FP64, t=50, s=100, cg_tol=1e-6, newton_tol=1e-7, cg_max_iter=3000)
    o32 = vl.Opts.make(precision=vl.FP32_REFINE, t=50, s=100, cg_tol=1e-6, newton_tol=1e-7, cg_max_iter=3000)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, m, o64)
    ex = fac.export()
    locs_v = P.locs[P.order]
    rows = fs.sample_rows(n, m, 120, 2)
    N_ref, A_ref, D_ref = fs.factor_rows(locs_v, rows, m, P.cov, P.sigma2, P.rho, P.nugget)
    assert np.array_equal(ex["N"][rows], N_ref)
    assert np.max(np.abs(ex["A"][rows] - A_ref)) < 1e-9 * max(1.0, np.max(np.abs(A_ref)))
    # D_i = sigma^2 - w^T w cancels where the neighbours nearly determine the point (D down to
    # ~4e-6 sigma^2 here): both sides' float64 rounding then bounds the absolute error near
    # eps sigma^2, so the bar is 1e-9 relative plus an absolute 1e-13 sigma^2
    assert np.all(np.abs(ex["D"][rows] - D_ref) <= 1e-9 * D_ref + 1e-13 * P.sigma2)

    out = {}
    for name, o in (("fp64", o64), ("mixed", o32)):
        st = fac.find_mode(P.lik, P.y, P.F, o)
        lml, stats = st.log_marglik(o, with_stats=True)
        mean, var = st.pred_var(P.test_locs, P.Fp, o)
        out[name] = (st.mode.copy(), lml, stats, st.mode_stats(), mean, var)
        st.close()
    b64, L64, s64, ms64, mu64, v64 = out["fp64"]
    b32, L32, s32, ms32, mu32, v32 = out["mixed"]
    assert np.max(np.abs(b32 - b64)) <= 1e-4 * np.max(np.abs(b64))
    assert abs(L32 - L64) <= 1e-4 * abs(L64)
    assert np.max(np.abs(mu32 - mu64)) <= 1e-4 * max(1.0, np.max(np.abs(mu64)))
    assert np.max(np.abs(v32 - v64) / v64) <= 1e-4
    assert len(mu64) == 10_000 and np.all(v64 > 0)
    assert ms32["true_relres_max"] <= 1e-6 and s32["probe_relres_max"] <= 1e-6
    assert ms64["true_relres_max"] <= 1e-6 and s64["probe_relres_max"] <= 1e-6
    assert s32["slq_stderr"] < 1e-3 * abs(L32)
    ctx.close()
