"""Serving form: a request loop over independent latent-GP problems.

Each request is a fresh problem (locations, responses, covariance parameters,
test points). Serving it runs the whole path on the device: the Vecchia factor
(Section 2.1), the Laplace mode (Eq. newton), L^VLA with the SLQ log-determinant
(Eqs. VLA_loss, def_SLQ) and the predictive means and variances (Algorithm simAlgo).

Execution model
---------------
* A slot is a library context with its own CUDA stream and a workspace large
  enough for the biggest admissible request. Slot contexts are made once and reused,
  so serving allocates no device memory after start-up.
* Admission is first-come first-served by HBM footprint: a free slot takes the
  first queued request that fits its workspace, once the estimated device footprint
  of the requests already running plus its own fits the budget. Slots may come in
  size classes (a few sized for the largest requests, many for small ones), so the
  order is first-come first-served within each class. A request that could never
  fit is rejected at once.
* Admitted requests run concurrently, each on its slot's stream from its own host
  thread (the library releases the interpreter lock), so their kernels overlap on
  the device as requests arrive and leave.
* Every kernel of the library is deterministic and requests share no device state,
  so a request's results are the same whether it runs alone or in the mix.
* Continuous batching (``batch_runner``): a slot that frees up takes the first queued
  request that fits and, in queue order, every further queued request with the same
  options while the group's footprint stays within the slot and the budget. The group
  runs as one merged block-diagonal system (``run_batch``: one launch of every kernel
  for all of its requests, each request with its own Newton iteration, PCG stopping
  rule and probes), so a request gets the same results alone and in a group up to the
  rounding of reductions taken over other block partitions.

The scheduler (admission, FIFO order, budget accounting) is plain host logic and
can be driven with any runner; ``run_request`` is the runner that calls the library.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Callable

import numpy as np


def footprint_bytes(n: int, m: int, t: int = 50, s: int = 100, n_test: int = 1000, k: int = 0) -> int:
    """Upper estimate of the device workspace one request needs (bytes): the factor
    (ELL of B and its transpose in float64 and float32, orders, levels), the state,
    and the largest phase, the simulation solves for predictive variances (float64
    and float32 Krylov blocks of up to 128 columns plus the refinement vectors), or
    the SLQ probe block with its float64 residual check. k > 0 adds the LRAC factor and its
    float copy."""
    def lead(c):
        return 1 if c == 1 else (c + 7) // 8 * 8
    ls, lt = lead(min(s, 128)), lead(t)
    factor = n * (200 + 40 * m)
    sim = n * ls * 132
    slq = n * lt * (4 * 10 + 8 * 4)   # float32 engine + probe blocks, float64 probe residual blocks
    test = n_test * (16 * m + 96)
    lrac = n * k * 12 + n * lt * 4 + 6 * k * k * 8 if k else 0
    return int(1.15 * (factor + max(sim, slq) + test + lrac)) + (32 << 20)


def batch_footprint_bytes(reqs) -> int:
    """Upper estimate of the workspace a merged group of requests needs (bytes): every
    member's own factor, plus the merged system (its factor, state and largest phase) as
    one request of the group's total size and largest m."""
    if not reqs:
        return 0
    o = reqs[0].opts
    N = sum(r.n for r in reqs)
    m = max(r.m for r in reqs)
    nt = sum(0 if r.test_locs is None else len(r.test_locs) for r in reqs)
    members = sum(int(1.15 * r.n * (200 + 40 * r.m)) for r in reqs)
    return footprint_bytes(N, m, o.get("t", 50), o.get("s", 100), nt) + members


@dataclasses.dataclass
class Request:
    rid: int
    locs: np.ndarray
    order: np.ndarray
    y: np.ndarray
    F: np.ndarray | None
    cov: int
    sigma2: float
    rho: float
    m: int
    lik: int
    test_locs: np.ndarray | None
    opts: dict
    arrival: float = 0.0          # server clock, seconds
    footprint: int = 0

    @property
    def n(self) -> int:
        return int(self.locs.shape[0])

    @classmethod
    def from_problem(cls, rid: int, P, opts: dict, arrival: float = 0.0) -> "Request":
        r = cls(rid=rid, locs=P.locs, order=P.order, y=P.y, F=P.F, cov=P.cov, sigma2=P.sigma2, rho=P.rho, m=P.m,
                lik=P.lik, test_locs=P.test_locs, opts=dict(opts), arrival=arrival)
        r.footprint = footprint_bytes(r.n, r.m, opts.get("t", 50), opts.get("s", 100),
                                      0 if P.test_locs is None else len(P.test_locs),
                                      opts.get("k", 0) if opts.get("precond", 0) == 2 else 0)
        return r


@dataclasses.dataclass
class Result:
    rid: int
    n: int
    slot: int
    t_arrival: float
    t_admit: float
    t_done: float
    lml: float = float("nan")
    mode: np.ndarray | None = None
    mean: np.ndarray | None = None
    var: np.ndarray | None = None
    stats: dict = dataclasses.field(default_factory=dict)
    error: str | None = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class Scheduler:
    """FIFO admission by footprint against a device-memory budget. ``group_footprint``
    (a list of requests -> bytes) prices the groups of continuous batching; by default a
    group costs the sum of its requests' footprints."""

    def __init__(self, budget_bytes: int, slot_capacity: int, group_footprint: Callable | None = None):
        self.budget = int(budget_bytes)
        self.capacity = int(slot_capacity)   # bytes the largest slot can hold
        self.group_footprint = group_footprint or (lambda reqs: sum(r.footprint for r in reqs))
        self.q: collections.deque[Request] = collections.deque()
        self.cv = threading.Condition()
        self.in_use = 0
        self.running = 0
        self.peak_in_use = 0
        self.peak_running = 0
        self.closed = False
        self.rejected: list[Request] = []

    def submit(self, req: Request, grouped: bool = False) -> bool:
        with self.cv:
            fp = self.group_footprint([req]) if grouped else req.footprint
            if fp > min(self.budget, self.capacity):
                self.rejected.append(req)
                return False
            self.q.append(req)
            self.cv.notify_all()
            return True

    def _first_fitting(self, capacity: int) -> int:
        for i, r in enumerate(self.q):
            if r.footprint <= capacity:
                return i
        return -1

    def acquire(self, timeout: float | None = None, capacity: int | None = None) -> Request | None:
        """Block until the first queued request that fits a slot of `capacity` bytes
        (default: the largest) also fits the budget (returning it, admitted), or the
        scheduler is closed and no queued request fits this slot (returning None)."""
        cap = self.capacity if capacity is None else int(capacity)
        deadline = None if timeout is None else time.perf_counter() + timeout
        with self.cv:
            while True:
                i = self._first_fitting(cap)
                if i >= 0 and self.in_use + self.q[i].footprint <= self.budget:
                    req = self.q[i]
                    del self.q[i]
                    self.in_use += req.footprint
                    self.running += 1
                    self.peak_in_use = max(self.peak_in_use, self.in_use)
                    self.peak_running = max(self.peak_running, self.running)
                    self.cv.notify_all()
                    return req
                if self.closed and i < 0:
                    return None
                left = None if deadline is None else deadline - time.perf_counter()
                if left is not None and left <= 0:
                    return None
                self.cv.wait(left)

    def acquire_group(self, capacity: int | None = None, max_group: int = 64,
                      timeout: float | None = None) -> tuple[list[Request], int]:
        """Continuous batching: block until the first queued request that fits a slot of
        `capacity` bytes, alone, also fits the budget; take it and then, in queue order,
        every further queued request with the same options while the group's footprint
        stays within the slot and the budget (at most max_group requests). Returns the
        group (removed from the queue, admitted) and its footprint, or ([], 0) once the
        scheduler is closed and no queued request fits this slot."""
        cap = self.capacity if capacity is None else int(capacity)
        deadline = None if timeout is None else time.perf_counter() + timeout
        with self.cv:
            while True:
                group: list[Request] = []
                fp = 0
                first_fits = False
                for r in self.q:
                    if len(group) >= max_group:
                        break
                    if group and r.opts != group[0].opts:
                        continue
                    f = self.group_footprint(group + [r])
                    if not group:
                        if f > cap:
                            continue           # not for this slot's size class
                        first_fits = True
                        if self.in_use + f > self.budget:
                            break              # first come, first served: the head waits for room
                        group.append(r)
                        fp = f
                    elif f <= cap and self.in_use + f <= self.budget:
                        group.append(r)
                        fp = f
                if group:
                    for r in group:
                        self.q.remove(r)
                    self.in_use += fp
                    self.running += len(group)
                    self.peak_in_use = max(self.peak_in_use, self.in_use)
                    self.peak_running = max(self.peak_running, self.running)
                    self.cv.notify_all()
                    return group, fp
                if self.closed and not first_fits:
                    return [], 0
                left = None if deadline is None else deadline - time.perf_counter()
                if left is not None and left <= 0:
                    return [], 0
                self.cv.wait(left)

    def release(self, req: Request):
        with self.cv:
            self.in_use -= req.footprint
            self.running -= 1
            self.cv.notify_all()

    def release_group(self, group: list[Request], footprint: int):
        with self.cv:
            self.in_use -= footprint
            self.running -= len(group)
            self.cv.notify_all()

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()


def run_batch(vl, ctx, reqs: list[Request]) -> list[dict]:
    """The whole path for a group of requests with the same options, merged into one
    block-diagonal system on one slot context (vl.Batch): factors, modes, L^VLA,
    predictive means and variances. A failure fails the whole group."""
    o = vl.Opts.make(**reqs[0].opts)
    facs, b = [], None
    try:
        for r in reqs:
            facs.append(ctx.build_factor(r.locs, r.order, r.cov, r.sigma2, r.rho, r.m, o))
        b = vl.Batch(ctx, facs)
        Fs = None if all(r.F is None for r in reqs) else [np.zeros(r.n) if r.F is None else r.F for r in reqs]
        modes, mstats = b.find_mode([r.lik for r in reqs], [r.y for r in reqs], Fs, o, with_stats=True)
        lml, lstats = b.log_marglik(o, with_stats=True)
        outs = [{"lml": float(lml[k]), "mode": modes[k], "stats": {"mode": mstats[k], "lml": lstats[k],
                                                                  "group": len(reqs)}}
                for k in range(len(reqs))]
        tl = [np.zeros((0, 2)) if r.test_locs is None else np.asarray(r.test_locs, np.float64) for r in reqs]
        if any(len(q) for q in tl):
            means, vars_ = b.pred_var(tl, None, o)
            for k, r in enumerate(reqs):
                if len(tl[k]):
                    outs[k]["mean"], outs[k]["var"] = means[k], vars_[k]
        return outs
    finally:
        if b is not None:
            b.close()
        for f in facs:
            f.close()


def run_request(vl, ctx, req: Request) -> dict:
    """The whole path for one request on one slot context (device work on its
    stream): factor, mode, L^VLA, predictive mean and variance."""
    o = vl.Opts.make(**req.opts)
    fac = ctx.build_factor(req.locs, req.order, req.cov, req.sigma2, req.rho, req.m, o)
    st = None
    try:
        st = fac.find_mode(req.lik, req.y, req.F, o)
        lml, stats = st.log_marglik(o, with_stats=True)
        out = {"lml": lml, "mode": st.mode, "stats": {"mode": st.mode_stats(), "lml": stats}}
        if req.test_locs is not None and len(req.test_locs):
            mean, var = st.pred_var(req.test_locs, None, o)
            out["mean"], out["var"] = mean, var
        return out
    finally:
        if st is not None:
            st.close()
        fac.close()


class Server:
    """Worker threads, one per slot, each owning one context (made by
    ``make_ctx(slot)``, or ``make_ctx(slot, capacity)`` when slots have capacities)
    and serving admitted requests with ``runner(ctx, req) -> dict``. ``slots`` is a
    count (every slot holds ``slot_capacity`` bytes) or a list of per-slot capacities."""

    def __init__(self, slots, budget_bytes: int, slot_capacity: int | None, make_ctx: Callable[..., object],
                 runner: Callable[[object, Request], dict] | None = None, clock: Callable[[], float] = time.perf_counter,
                 batch_runner: Callable[[object, list], list] | None = None, max_group: int = 64,
                 group_footprint: Callable | None = None):
        caps = [int(slot_capacity)] * slots if isinstance(slots, int) else [int(c) for c in slots]
        if (runner is None) == (batch_runner is None):
            raise ValueError("give exactly one of runner and batch_runner")
        self.caps = caps
        self.sched = Scheduler(budget_bytes, max(caps), group_footprint)
        self.make_ctx, self.runner, self.clock = make_ctx, runner, clock
        self.batch_runner, self.max_group = batch_runner, int(max_group)
        self.groups: list[int] = []          # sizes of the groups served (continuous batching)
        self._sized = not isinstance(slots, int)
        self.results: list[Result] = []
        self._lock = threading.Lock()
        self._ready = threading.Barrier(len(caps) + 1)
        self.threads = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(len(caps))]
        self.t0 = 0.0
        self.errors: list[str] = []

    def start(self):
        for th in self.threads:
            th.start()
        self._ready.wait()          # every slot context exists before the clock starts
        if self.errors:             # a slot without a context would leave its requests unserved
            self.sched.close()
            for th in self.threads:
                th.join()
            raise RuntimeError("slot context creation failed: " + "; ".join(self.errors))
        self.t0 = self.clock()
        return self

    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, req: Request, stamp: bool = True) -> bool:
        if stamp:
            req.arrival = self.now()
        ok = self.sched.submit(req, grouped=self.batch_runner is not None)
        if not ok:
            with self._lock:
                self.results.append(Result(req.rid, req.n, -1, req.arrival, req.arrival, req.arrival,
                                           error="rejected: footprint above the budget"))
        return ok

    def _worker(self, slot: int):
        try:
            ctx = self.make_ctx(slot, self.caps[slot]) if self._sized else self.make_ctx(slot)
        except Exception as e:          # noqa: BLE001 - reported to the caller
            self.errors.append(f"slot {slot}: {e}")
            self._ready.wait()
            return
        self._ready.wait()
        if self.batch_runner is not None:
            self._serve_groups(slot, ctx)
        while self.batch_runner is None:
            req = self.sched.acquire(capacity=self.caps[slot])
            if req is None:
                break
            t_admit = self.now()
            res = Result(req.rid, req.n, slot, req.arrival, t_admit, t_admit)
            try:
                out = self.runner(ctx, req)
                res.lml = out.get("lml", float("nan"))
                res.mode, res.mean, res.var = out.get("mode"), out.get("mean"), out.get("var")
                res.stats = out.get("stats", {})
            except Exception as e:      # noqa: BLE001 - recorded per request
                res.error = f"{type(e).__name__}: {e}"
            res.t_done = self.now()
            self.sched.release(req)
            with self._lock:
                self.results.append(res)
        close = getattr(ctx, "close", None)
        if close:
            close()

    def _serve_groups(self, slot: int, ctx):
        while True:
            group, fp = self.sched.acquire_group(capacity=self.caps[slot], max_group=self.max_group)
            if not group:
                return
            t_admit = self.now()
            res = [Result(r.rid, r.n, slot, r.arrival, t_admit, t_admit) for r in group]
            try:
                outs = self.batch_runner(ctx, group)
                for x, out in zip(res, outs):
                    x.lml = out.get("lml", float("nan"))
                    x.mode, x.mean, x.var = out.get("mode"), out.get("mean"), out.get("var")
                    x.stats = out.get("stats", {})
            except Exception as e:      # noqa: BLE001 - recorded for every request of the group
                for x in res:
                    x.error = f"{type(e).__name__}: {e}"
            t_done = self.now()
            self.sched.release_group(group, fp)
            with self._lock:
                for x in res:
                    x.t_done = t_done
                    self.results.append(x)
                self.groups.append(len(group))

    def drain(self):
        """Stop taking requests once the queue is empty and wait for the workers."""
        self.sched.close()
        for th in self.threads:
            th.join()
        return sorted(self.results, key=lambda r: r.rid)


def latency_summary(results: list[Result], wall_s: float) -> dict:
    ok = [r for r in results if r.error is None]
    lat = np.array([r.latency for r in ok]) * 1e3
    svc = np.array([r.t_done - r.t_admit for r in ok]) * 1e3
    wait = np.array([r.t_admit - r.t_arrival for r in ok]) * 1e3
    q = (lambda a, p: float(np.percentile(a, p)) if len(a) else None)
    return {
        "requests": len(results), "completed": len(ok), "failed": len(results) - len(ok),
        "p50_latency_ms": q(lat, 50), "p99_latency_ms": q(lat, 99), "max_latency_ms": q(lat, 100),
        "p50_service_ms": q(svc, 50), "p99_service_ms": q(svc, 99), "p50_queue_ms": q(wait, 50),
        "p99_queue_ms": q(wait, 99), "throughput_rps": len(ok) / wall_s if wall_s > 0 else None,
        "points_per_s": float(sum(r.n for r in ok) / wall_s) if wall_s > 0 else None,
    }


def gpu_slots(vl, device: int, ws_bytes: int | None = None) -> Callable[..., object]:
    """Slot factory: one library context per slot on its own CUDA stream, with a
    workspace (ws_bytes, or the slot's capacity) taken from PyTorch's device memory."""
    import torch

    def make(slot: int, capacity: int | None = None):
        torch.cuda.set_device(device)
        stream = torch.cuda.Stream(device)
        ctx = vl.Context(device, ws_bytes=int(capacity or ws_bytes), stream=stream)
        ctx._slot_stream = stream      # keep the stream alive with the context
        return ctx
    return make
