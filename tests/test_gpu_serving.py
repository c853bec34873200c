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
