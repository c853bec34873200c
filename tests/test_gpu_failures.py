"""Failure paths of the library on the GPU, made without faulting or hanging the device.

* VL_ERR_TIMEOUT: every device-side spin of the library (the software grid barriers of the
  triangular solves, the level-schedule walk) is a bounded wait; when one runs out it records
  the error, every other wait of the launch gives up, and the call returns VL_ERR_TIMEOUT.
  A probe waits on a flag that nothing sets (vl_ctx_wait_probe); the real walk is run under a
  limit of one cycle. In both cases the context keeps working afterwards.
* VL_ERR_NOT_CONVERGED: PCG capped at a few iterations (float64 Newton solves, the SLQ probe
  solves, mixed-precision refinement).
* VL_ERR_OOM: a workspace too small for the factor; nothing leaks.
* VL_ERR_INVALID_ARG: responses outside the likelihood's support, NaN or infinite values.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import geometry

pytestmark = pytest.mark.gpu

TIMEOUT, NOT_CONVERGED, OOM, INVALID = 5, 4, 2, 1


@pytest.fixture(scope="module")
def vl():
    import paper_2310_12000_gb300 as vl
    vl.library()
    return vl


def test_wait_probe_times_out_and_the_context_recovers(vl):
    ctx = vl.Context(0, ws_bytes=256 << 20)
    ctx.set_wait_limit(2_000_000)            # about 1 ms
    for _ in range(2):
        with pytest.raises(vl.VLError) as e:
            ctx.wait_probe()
        assert e.value.status == TIMEOUT and "timed out" in str(e.value)
    ctx.set_wait_limit(0)
    with pytest.raises(vl.VLError):
        ctx.set_wait_limit(-1)
    P = wl.make_problem("c1_n2000", n=1500)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    assert np.array_equal(fac.export()["N"], geometry.knn_prev(P.locs[P.order], P.m))
    ctx.close()


def test_real_wait_runs_out_under_a_one_cycle_limit(vl):
    """The level-schedule walk waits on rows of earlier levels (a chain of about 250 levels
    here); with a limit of one cycle the first wait that is not satisfied at once gives up."""
    ctx = vl.Context(0, ws_bytes=1 << 30)
    P = wl.make_problem("c1_n2000", n=50_000)
    ctx.set_wait_limit(1)
    with pytest.raises(vl.VLError) as e:
        ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    assert e.value.status == TIMEOUT and "level schedule" in str(e.value)
    assert ctx.mem()[0] < 1 << 20                      # the failed build returned its blocks
    ctx.set_wait_limit(0)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    ex = fac.export()
    rows = np.random.default_rng(0).choice(P.n, 100, replace=False)
    assert np.array_equal(ex["N"][rows], geometry.knn_prev_rows(P.locs[P.order], P.m, rows))
    info = fac.info()
    assert info["nlev_fwd"] == int(ex["lev_fwd"].max()) + 1
    ctx.close()


def test_capped_pcg_is_not_converged(vl):
    ctx = vl.Context(0, ws_bytes=1 << 30)
    P = wl.make_problem("c1_n2000", n=3000)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    with pytest.raises(vl.VLError) as e:                          # float64 Newton solves
        fac.find_mode(P.lik, P.y, P.F, vl.Opts.make(cg_max_iter=2, cg_tol=1e-10))
    assert e.value.status == NOT_CONVERGED and "cg_max_iter" in str(e.value)
    with pytest.raises(vl.VLError) as e:                          # mixed-precision refinement
        fac.find_mode(P.lik, P.y, P.F, vl.Opts.make(precision=vl.FP32_REFINE, cg_max_iter=1, cg_tol=1e-8))
    assert e.value.status == NOT_CONVERGED
    st = fac.find_mode(P.lik, P.y, P.F, vl.Opts.make(cg_tol=1e-10))
    with pytest.raises(vl.VLError) as e:                          # SLQ probe solves
        st.log_marglik(vl.Opts.make(t=8, cg_max_iter=3, cg_tol=1e-8))
    assert e.value.status == NOT_CONVERGED
    lml = st.log_marglik(vl.Opts.make(t=8, cg_tol=1e-8))         # and the state still works
    assert np.isfinite(lml)
    ctx.close()


def test_workspace_exhaustion_is_reported_and_nothing_leaks(vl):
    ctx = vl.Context(0, ws_bytes=4 << 20)
    base = ctx.mem()[0]
    P = wl.make_problem("c1_n2000", n=20_000)
    with pytest.raises(vl.VLError) as e:
        ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    assert e.value.status == OOM and "workspace exhausted" in str(e.value)
    assert ctx.mem()[0] == base
    small = wl.make_problem("c1_n2000", n=300)
    fac = ctx.build_factor(small.locs, small.order, small.cov, small.sigma2, small.rho, small.m)
    assert np.array_equal(fac.export()["N"], geometry.knn_prev(small.locs[small.order], small.m))
    fac.close()
    assert ctx.mem()[0] == base
    ctx.close()


def test_responses_outside_the_support_are_refused(vl):
    ctx = vl.Context(0, ws_bytes=256 << 20)
    P = wl.make_problem("c1_n2000", n=800)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m)
    opts = vl.Opts.make(cg_tol=1e-8)
    cases = [(vl.LIK_BERNOULLI_LOGIT, 17, np.nan, None), (vl.LIK_BERNOULLI_LOGIT, 3, 2.0, None),
             (vl.LIK_POISSON_LOG, 40, -1.0, None), (vl.LIK_POISSON_LOG, 41, 1.5, None),
             (vl.LIK_GAMMA_LOG, 5, 0.0, None), (vl.LIK_POISSON_LOG, 0, np.inf, None),
             (vl.LIK_BERNOULLI_LOGIT, None, None, 9)]
    for lik, bad_y, val, bad_F in cases:
        y = (P.y if lik == vl.LIK_BERNOULLI_LOGIT else P.y + 1.0).copy()
        F = np.zeros(P.n)
        if bad_y is not None:
            y[bad_y] = val
        if bad_F is not None:
            F[bad_F] = np.nan
        o = vl.Opts.make(cg_tol=1e-8, lik_shape=3.0)
        with pytest.raises(vl.VLError) as e:
            fac.find_mode(lik, y, F, o)
        assert e.value.status == INVALID, (lik, bad_y, val)
        assert f"y[{bad_y if bad_y is not None else bad_F}]" in str(e.value)
    st = fac.find_mode(P.lik, P.y, P.F, opts)
    assert np.all(np.isfinite(st.mode))
    ctx.close()
