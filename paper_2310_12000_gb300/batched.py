"""Batched form: many independent latent-GP problems of uneven size solved together.

Each problem is a full L^VLA evaluation: Vecchia factor (Section 2.1), Newton mode
(Eq. newton) and the SLQ log-determinant (Eqs. VLA_loss, def_SLQ), float32 Krylov
solves with float64 refinement.

``run_merged`` merges the problems into one block-diagonal system (``vl.Batch``): one
launch of every kernel serves all problems, a triangular solve walks as many levels as
the deepest problem, and each problem keeps its own Newton iteration, stopping rules and
probes. ``run_batch`` spreads the problems over slot contexts on separate CUDA streams
(see ``serving``) instead. Results do not depend on the grouping.
"""
from __future__ import annotations

import time

import numpy as np

from . import serving


def run_merged(vl, problems, opts: dict | None = None, device: int = 0, steps: int = 2, warmup: int = 1,
               ws_bytes: int | None = None) -> dict:
    """Merged form: builds every factor and the batch once (neighbours, levels; not timed),
    then times `steps` evaluations of every problem (factor rows for the covariance
    parameters, Newton modes, SLQ and L^VLA) on the device with CUDA events."""
    import torch
    opts = dict(opts or dict(precision=1, t=50, cg_tol=1e-6, newton_tol=1e-7))
    n_tot = sum(P.n for P in problems)
    ws = ws_bytes or int(min(torch.cuda.mem_get_info(device)[0] * 0.6, max(8 << 30, n_tot * 20000)))
    ctx = vl.Context(device, ws_bytes=ws)
    o = vl.Opts.make(**opts)
    t0 = time.perf_counter()
    facs = [ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, o) for P in problems]
    b = vl.Batch(ctx, facs)
    build_s = time.perf_counter() - t0
    liks = [P.lik for P in problems]
    ys = [P.y for P in problems]
    Fs = [P.F for P in problems]

    def evaluation():
        for P, f in zip(problems, facs):
            f.refit(P.sigma2, P.rho, o)
        b.refresh()
        modes, mstats = b.find_mode(liks, ys, Fs, o, with_stats=True)
        lml, lstats = b.log_marglik(o, with_stats=True)
        return modes, mstats, lml, lstats

    for _ in range(warmup):
        evaluation()
    stream = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    e0.record(stream)
    for _ in range(steps):
        modes, mstats, lml, lstats = evaluation()
    e1.record(stream)
    torch.cuda.synchronize(device)
    sec = e0.elapsed_time(e1) / 1000.0 / steps
    info = b.info()
    out = {
        "problems": len(problems), "form": "merged", "n_total": n_tot, "levels_fwd": info["nlev_fwd"],
        "levels_bwd": info["nlev_bwd"], "build_s": build_s, "seconds_per_batch": sec,
        "evals_per_s": len(problems) / sec, "points_per_s": n_tot / sec, "steps": steps,
        "max_true_relres": float(max(max(s["true_relres_max"] for s in mstats),
                                     max(s["probe_relres_max"] for s in lstats))),
        "newton_iters_max": int(max(s["newton_iters"] for s in mstats)),
        "slq_cg_iters_max": int(max(s["cg_iters_max"] for s in lstats)),
        "lml": [float(v) for v in np.asarray(lml)],
    }
    b.close()
    for f in facs:
        f.close()
    ctx.close()
    return out


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
