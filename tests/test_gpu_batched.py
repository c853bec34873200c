"""Batched form on the GPU: every problem of an uneven batch solved on slot contexts
gives the same L^VLA as the same problem solved alone."""
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def test_batch_matches_single_runs():
    import paper_2310_12000_gb300 as vl
    from paper_2310_12000_gb300 import batched, serving
    vl.library()
    probs = [wl.batched_problem(i, n=n) for i, n in enumerate([5000, 12000, 7000, 20000, 5500, 9000])]
    opts = dict(precision=1, t=16, cg_tol=1e-6, newton_tol=1e-7)
    out = batched.run_batch(vl, probs, slots=3, opts=opts)
    assert out["failed"] == 0, out["errors"]
    assert out["max_true_relres"] <= 1e-6
    for i, P in enumerate(probs):
        req = serving.Request.from_problem(i, P, opts)
        ctx = vl.Context(0, ws_bytes=req.footprint)
        alone = serving.run_request(vl, ctx, req)
        ctx.close()
        assert alone["lml"] == out["lml"][i]
