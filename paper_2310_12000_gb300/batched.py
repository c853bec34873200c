"""Batched form: many independent latent-GP problems of uneven size solved together.

Each problem is a full L^VLA evaluation: Vecchia factor (Section 2.1), Newton mode
(Eq. newton) and the SLQ log-determinant (Eqs. VLA_loss, def_SLQ), float32 Krylov
solves with float64 refinement. The problems are spread over slot contexts, each
on its own CUDA stream (see ``serving``): while one problem waits on its level
barriers or host read-backs the others keep the device busy, and small problems
take small parts of the device (a t = 1 solve of a small system is one block, a
block solve one thread-block cluster). Results do not depend on the grouping.
"""
from __future__ import annotations

import time

from . import serving


def run_batch(vl, problems, slots: int = 16, opts: dict | None = None, device: int = 0) -> dict:
    """Solves every problem once; returns throughput and per-problem results."""
    opts = dict(opts or dict(precision=1, t=50, cg_tol=1e-6, newton_tol=1e-7))
    reqs = [serving.Request.from_problem(i, P, opts) for i, P in enumerate(problems)]
    for r in reqs:
        r.test_locs = None
    cap = max(r.footprint for r in reqs)
    srv = serving.Server(slots=slots, budget_bytes=slots * cap, slot_capacity=cap,
                         make_ctx=serving.gpu_slots(vl, device, cap),
                         runner=lambda ctx, req: serving.run_request(vl, ctx, req)).start()
    t0 = time.perf_counter()
    for r in reqs:
        srv.submit(r)
    res = srv.drain()
    wall = time.perf_counter() - t0
    ok = [r for r in res if r.error is None]
    relres = [r.stats.get("mode", {}).get("true_relres_max", 0.0) for r in ok]
    return {
        "problems": len(problems), "completed": len(ok), "failed": len(res) - len(ok), "slots": slots,
        "wall_s": wall, "evals_per_s": len(ok) / wall, "points_per_s": float(sum(r.n for r in ok) / wall),
        "max_true_relres": float(max(relres)) if relres else None,
        "peak_concurrent": srv.sched.peak_running,
        "lml": [r.lml for r in res], "errors": [r.error for r in res if r.error][:3],
    }
