"""Serving form on the GPU: requests served concurrently on slot contexts give the
same results as each request served alone, and the admission footprint estimate
bounds the device memory a request actually uses."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

OPTS = dict(precision=1, t=16, s=32, cg_tol=1e-6, newton_tol=1e-7)
SIZES = [3000, 12000, 5000, 20000, 8000, 2000]


@pytest.fixture(scope="module")
def vl():
    import paper_2310_12000_gb300 as vl
    vl.library()
    return vl


def _requests(serving):
    return [serving.Request.from_problem(i, wl.serving_problem(i, n=n), OPTS) for i, n in enumerate(SIZES)]


def _serve(vl, serving, reqs, slots):
    ws = max(r.footprint for r in reqs)
    srv = serving.Server(slots=slots, budget_bytes=slots * ws, slot_capacity=ws,
                         make_ctx=serving.gpu_slots(vl, 0, ws),
                         runner=lambda ctx, req: serving.run_request(vl, ctx, req)).start()
    for r in reqs:
        srv.submit(r)
    return srv, srv.drain()


def test_results_identical_alone_and_in_mix(vl):
    from paper_2310_12000_gb300 import serving
    srv_mix, mix = _serve(vl, serving, _requests(serving), slots=3)
    assert all(r.error is None for r in mix), [r.error for r in mix]
    assert srv_mix.sched.peak_running >= 2          # requests really overlapped
    _, alone = _serve(vl, serving, _requests(serving), slots=1)
    for a, b in zip(mix, alone):
        assert a.rid == b.rid and b.error is None
        assert a.lml == b.lml
        assert np.array_equal(a.mode, b.mode)
        assert np.array_equal(a.mean, b.mean) and np.array_equal(a.var, b.var)
        assert a.stats["mode"]["true_relres_max"] <= 1e-6


def test_footprint_estimate_bounds_peak_use(vl):
    from paper_2310_12000_gb300 import serving
    for i, n in enumerate([4000, 30000]):
        req = serving.Request.from_problem(i, wl.serving_problem(i, n=n), dict(OPTS, t=50, s=100))
        ctx = vl.Context(0, ws_bytes=req.footprint)
        serving.run_request(vl, ctx, req)
        _, peak = ctx.mem()
        ctx.close()
        assert peak <= req.footprint, (n, peak, req.footprint)


def _close(a, b, tol):
    return np.max(np.abs(a - b)) <= tol * max(1.0, np.max(np.abs(b)))


def test_continuous_batching_matches_requests_alone(vl):
    """Requests served in merged groups (continuous batching, run_batch) against each request
    served alone (run_request): mixed precision within the stated 1e-4 on L^VLA, the mode and
    the predictive mean and variance, every refined residual <= 1e-6; groups of several
    requests really formed."""
    from paper_2310_12000_gb300 import serving
    reqs = _requests(serving)
    cap = serving.batch_footprint_bytes(reqs)
    srv = serving.Server(slots=1, budget_bytes=cap, slot_capacity=cap, make_ctx=serving.gpu_slots(vl, 0, cap),
                         batch_runner=lambda ctx, g: serving.run_batch(vl, ctx, g)).start()
    for r in reqs:
        srv.submit(r)
    grouped = srv.drain()
    assert max(srv.groups) > 1, srv.groups
    _, alone = _serve(vl, serving, _requests(serving), slots=1)
    for a, b in zip(grouped, alone):
        assert a.rid == b.rid and a.error is None and b.error is None, (a.error, b.error)
        assert abs(a.lml - b.lml) <= 1e-4 * abs(b.lml)
        assert _close(a.mode, b.mode, 1e-4)
        assert _close(a.mean, b.mean, 1e-4)
        assert np.max(np.abs(a.var - b.var) / b.var) <= 1e-4
        assert a.stats["mode"]["true_relres_max"] <= 1e-6 and a.stats["lml"]["probe_relres_max"] <= 1e-6


def test_merged_group_equals_alone_fp64(vl):
    """The float64 path: a merged group gives each request what it gets alone within 1e-9."""
    from paper_2310_12000_gb300 import serving
    o = dict(precision=0, t=12, s=16, cg_tol=1e-12, newton_tol=1e-10, cg_max_iter=3000)
    reqs = [serving.Request.from_problem(i, wl.serving_problem(i, n=n), o) for i, n in enumerate([2500, 6000, 1000])]
    cap = serving.batch_footprint_bytes(reqs)
    ctx = vl.Context(0, ws_bytes=cap)
    outs = serving.run_batch(vl, ctx, reqs)
    _, peak = ctx.mem()
    assert peak <= cap
    for r, g in zip(reqs, outs):
        a = serving.run_request(vl, ctx, r)
        assert abs(g["lml"] - a["lml"]) <= 1e-9 * abs(a["lml"])
        assert _close(g["mode"], a["mode"], 1e-9) and _close(g["mean"], a["mean"], 1e-9)
        assert np.max(np.abs(g["var"] - a["var"]) / a["var"]) <= 1e-9
    ctx.close()
