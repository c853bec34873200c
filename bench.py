"""Benchmark of the iterative Vecchia-Laplace hot path on GB300.

One step = one evaluation of the Vecchia-Laplace negative log-marginal likelihood
at fixed covariance parameters and fixed locations: the Vecchia factor rows (A_i,
D_i), Newton's mode with PCG solves, the SLQ probe solves and the L^VLA
assembly. Neighbour sets and level schedules depend only on the locations; they
are built once before timing and reported separately (graph_ms).

Workload (default): n = 1,000,000 points of a 1250 x 1000 grid over the unit
square with 20% removed in rectangular gaps, Matern-1.5 covariance (sigma2 = 1,
range 0.02), m = 20, Poisson-log responses with offset 1.0, t = 50 Rademacher
probes, VADU preconditioner, float32 Krylov path with float64 refinement.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Two more legs run on rank 0 of a single-GPU run, after the timed steps:
* batched: 256 independent problems (n log-uniform in [5e3, 5e4], m in {10, 20,
  30}, exponential covariance, Bernoulli-logit), mode + L^VLA each, spread over
  slot contexts on separate streams; reported as evaluations/s.
* serving: a Poisson stream of fresh problems at 50 requests/s (n log-uniform in
  [1e3, 2e5], Matern-1.5, Bernoulli or Poisson, mode + L^VLA + predictive
  variances at 1000 points) admitted by device-memory footprint, each on a slot
  context of its own with the slots' work overlapping on the device (`--serve-form
  groups`: a free slot merges every queued request that fits into one block-diagonal
  system instead); reported as p50 / p99 latency (arrival to completion), service
  time and throughput, with the arrival window stated.

Multi-GPU (torchrun, one rank per GPU): independent replicas, each rank solving its
own seeded problem of the same shape (weak scaling); no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "n=1M log-marglik evals/s (mixed vs FP64) at stated err; PCG HBM GB/s; p99 latency"
UNIT = "evals/s"
WORKLOAD = "c3_grid1m"
CPU_SAMPLE_N = 20000


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# FP64 ALU peak from unit counts and clocks: 152 SMs x 2 FP64 FMA lanes per SM per clock
# (1:64 of the 128 FP32 lanes) x 2 flops x 2070 MHz = 1.26 TFLOP/s (nominal 1.25).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def derived_metrics(prof: dict, n: int, m: int, ms_per_step: float, graph_ms: float) -> dict:
    """Figures derived from measured times only: the factor rows (a4) as an FP64 ALU-bound
    kernel (per row m^3/3 + 2m^2 + 2m flops: Cholesky of Sigma_N, two triangular solves,
    w^T w; the covariance evaluations are not counted) and the evaluation rate with the
    neighbour search and level schedules (one build_factor) included in every evaluation."""
    out = {"evals_per_s_incl_graph": 1000.0 / (ms_per_step + graph_ms) if ms_per_step + graph_ms > 0 else None}
    ent = (prof or {}).get("factor") or {}
    if ent.get("launches") and ent.get("ms", 0) > 0:
        flops_row = m ** 3 / 3 + 2 * m * m + 2 * m
        flops = _nnz(n, m) / max(m, 1) * flops_row if m else 0.0   # rows with fewer neighbours counted pro rata
        avg_s = ent["ms"] / ent["launches"] / 1000.0
        achieved = flops / avg_s / 1e12
        out["factor_roofline"] = {"bound": "alu", "dtype": "f64", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                                  "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                                  "peak_source": "152 SMs x 2 FP64 FMA lanes x 2 flops x 2070 MHz (no measured "
                                                 "FP64 peak)", "flops_per_row": flops_row,
                                  "avg_launch_ms": avg_s * 1000.0}
    return out


def newton_summary(ms: dict) -> dict:
    """Newton steps, PCG iterations (all refinement passes) and iterations per step of one
    mode computation, from the state's statistics."""
    steps = int(ms.get("newton_iters") or 0)
    its = int(ms.get("cg_iters_total") or 0)
    return {"steps": steps, "cg_iters_total": its, "cg_iters_per_step": its / steps if steps else None,
            "pcg_solves": ms.get("cg_calls"), "refine_passes": ms.get("refine_steps"),
            "true_relres": ms.get("true_relres_max")}


def _nnz(n: int, m: int) -> int:
    return sum(min(k, m) for k in range(min(n, m))) + max(0, n - m) * m


def algorithmic_bytes(cls: str, n: int, m: int, t: int, e: int, k: int = 0) -> float:
    """Bytes one launch of kernel class `cls` must move (each operand once)."""
    nnz = _nnz(n, m)
    vec = n * t * e
    if cls == "woodbury":       # L read for L^T(WR) and again for L V; R read twice, W, Z written
        return 2 * n * k * e + 3 * vec + n * e
    if cls == "sptrsv_fwd":     # ELL (idx + val), task list, rhs, row scale, solution
        return nnz * (4 + e) + 4 * n + vec + n * e + vec
    if cls == "sptrsv_bwd":     # CSR (idx + val + row pointers), task list, rhs, solution
        return nnz * (4 + e) + 4 * (n + 1) + 4 * n + vec + vec
    if cls == "spmv_B":         # ELL, X, row scale, Y
        return nnz * (4 + e) + vec + n * e + vec
    if cls == "spmv_Bt":        # CSR, Y, X, diagonal, Z
        return nnz * (4 + e) + 4 * (n + 1) + 3 * vec + n * e
    if cls == "coldot":
        return 2 * vec
    if cls == "pcg_update":     # two kernels per step, alternating: u, h, r, v -> u, r (6 vectors); z, h -> h (3)
        return 4.5 * vec
    return float("nan")


def _kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("kernels.cuh", "engine.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2310_12000_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(cls: str, t: int):
    """Per-launch DRAM bytes from the committed ncu summary, if it matches the kernels."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_hash") != _kernel_hash():
        return None
    ent = d.get("per_launch_bytes", {}).get(f"{cls}/t={t}")
    return ent


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        if not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle timing
def _oracle_eval_seconds(n_sub: int, seed: int) -> tuple[float, float]:
    """One oracle LML evaluation (factor rows, Newton with sparse LU, exact log-det)
    on the same recipe at n_sub points; neighbours built before timing."""
    import workloads as wl
    from oracle import laplace as la
    P = wl.make_problem(WORKLOAD, seed=seed, n=n_sub)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    t0 = time.perf_counter()
    f = la.refit(f, P.sigma2, P.rho, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik)
    L, _ = la.lml_exact(f, md)
    return time.perf_counter() - t0, L


ARM_PARTS = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1",
             "0xd49": "Arm Neoverse N2", "0xd8e": "Arm Neoverse N3", "0xd84": "Arm Neoverse V3"}


def cpu_model() -> str:
    part = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key == "model name":
                return line.split(":", 1)[1].strip()
            if key == "cpu part" and part is None:
                part = line.split(":", 1)[1].strip()
    except OSError:
        pass
    if part:
        return f"{ARM_PARTS.get(part.lower(), 'Arm')} (CPU part {part})"
    import platform
    return platform.processor() or platform.machine()


def _oracle_seconds(threads: int, steps: int) -> list:
    """Seconds per oracle evaluation in a child process with `threads` BLAS/OpenMP threads."""
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench, json; "
            f"r = [bench._oracle_eval_seconds({CPU_SAMPLE_N}, 1) for _ in range({steps})]; "
            f"print(json.dumps([x[0] for x in r]))")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-400:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline(n_full: int, steps: int = 1) -> dict:
    """The oracle timed on this host in child processes, single-threaded and with every core
    available to its BLAS (SuperLU itself is single-threaded)."""
    cores = os.cpu_count() or 1
    try:
        one = statistics.median(_oracle_seconds(1, steps))
        allc = statistics.median(_oracle_seconds(cores, steps))
    except RuntimeError as exc:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": str(exc)}
    best, used = (one, 1) if one <= allc else (allc, cores)
    scale = CPU_SAMPLE_N / n_full
    return {"value": (1.0 / best) * scale, "unit": UNIT, "cores": used, "kind": "oracle",
            "single_thread": {"value": scale / one, "seconds_per_eval_at_sample": one, "cores": 1},
            "all_cores": {"value": scale / allc, "seconds_per_eval_at_sample": allc, "cores": cores},
            "host": {"nproc": cores, "cpu_model": cpu_model()},
            "sample": f"one LML evaluation (factor rows + Newton with sparse-LU solves + exact log-det) of the "
                      f"same grid-with-gaps recipe at n={CPU_SAMPLE_N}, scaled to n={n_full} by n_sample/n "
                      f"(linear; flatters the CPU since sparse LU grows faster than n); value = the faster of "
                      f"1 thread and {cores} BLAS threads"}


# ----------------------------------------------------------------------------- batched / serving legs
def _gen_serving(i):
    import workloads as wl
    return wl.serving_problem(i)


def _gen_batched(i):
    import workloads as wl
    return wl.batched_problem(i)


def pregenerate(kind: str, count: int, procs: int = 12):
    """Draws the problems of a leg in a spawned process pool (inputs, not timed)."""
    import multiprocessing as mp
    fn = _gen_serving if kind == "serving" else _gen_batched
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(fn, range(count), chunksize=4)


def serving_leg(vl, problems, arrivals, duration: float, slots: int, device: int, small: int = 0,
                form: str = "slots", group_slots: int = 2, group_gb: float = 60.0) -> dict:
    """The serving stream. form "groups": continuous batching, `group_slots` slot contexts of
    group_gb GiB each, a free slot merging every queued request that fits into one
    block-diagonal system; form "slots": one request per slot context, `slots` of them."""
    import numpy as np
    from paper_2310_12000_gb300 import serving
    opts = dict(precision=1, t=50, s=100, cg_tol=1e-6, newton_tol=1e-7)
    reqs = [serving.Request.from_problem(i, P, opts) for i, P in enumerate(problems)]
    if form == "groups":
        cap = int(group_gb * (1 << 30))
        caps = [cap] * group_slots
        srv = serving.Server(slots=caps, budget_bytes=sum(caps), slot_capacity=None,
                             make_ctx=serving.gpu_slots(vl, device), max_group=256,
                             group_footprint=serving.batch_footprint_bytes,
                             batch_runner=lambda ctx, g: serving.run_batch(vl, ctx, g)).start()
        classes = {f"{group_gb:g} GiB merged-group slots": group_slots}
    else:
        # slot classes: `small` slots sized for n <= 6e4, the rest for the largest requests (n = 2e5)
        big = slots - small
        caps = [serving.footprint_bytes(200_000, 20)] * big + [serving.footprint_bytes(60_000, 20)] * small
        srv = serving.Server(slots=caps, budget_bytes=sum(caps), slot_capacity=None,
                             make_ctx=serving.gpu_slots(vl, device),
                             runner=lambda ctx, req: serving.run_request(vl, ctx, req)).start()
        classes = {"n<=2e5": big, "n<=6e4": small}
    for r, t in zip(reqs, arrivals):
        now = srv.now()
        if t > now:
            time.sleep(t - now)
        srv.submit(r)
    res = srv.drain()
    wall = srv.now()
    out = serving.latency_summary(res, wall)
    out.update({"form": "continuous batching (merged groups)" if form == "groups" else "one request per slot",
                "offered_rps": len(arrivals) / duration, "arrival_window_s": duration, "slots": len(caps),
                "slot_classes": classes,
                "groups": ({"count": len(srv.groups), "mean": float(np.mean(srv.groups)), "max": max(srv.groups)}
                           if srv.groups else None),
                "note": (f"arrivals offered for {duration:g} s at {len(arrivals) / duration:.1f} req/s, then "
                         f"drained: p50/p99 latency include the queueing behind that backlog; "
                         f"p50/p99_service_ms exclude it"),
                "peak_concurrent": srv.sched.peak_running, "wall_s": wall,
                "mean_n": float(np.mean([r.n for r in reqs])) if reqs else None,
                "max_true_relres": max((r.stats.get("mode", {}).get("true_relres_max", 0.0) for r in res
                                        if r.error is None), default=None),
                "errors": [r.error for r in res if r.error][:3],
                "workload": "Poisson arrivals; per request n log-uniform in [1e3, 2e5], uniform locations, "
                            "Matern-1.5 range U[0.02, 0.2], m=20, Bernoulli or Poisson (p=1/2), mode + L^VLA "
                            "(t=50) + predictive mean/variance at 1000 points (s=100), float32 + float64 "
                            "refinement; admission FIFO by device-memory footprint"})
    return out


# ----------------------------------------------------------------------------- distributed
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_throughput(elapsed_s: float, steps: int) -> tuple[float, float]:
    """Replicas-only aggregation: every rank solved `steps` problems of its own in
    elapsed_s seconds; the job took the slowest rank's time, and the whole-job
    throughput counts all ranks' problems. Returns (max elapsed, evals/s)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    if ws > 1:
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([elapsed_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_s = float(t.item())
    return elapsed_s, ws * steps / elapsed_s


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    n_full = 1_000_000
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench, json; "
            f"[bench._oracle_eval_seconds({CPU_SAMPLE_N}, 1) for _ in range({args.warmup})]; "
            f"r = [bench._oracle_eval_seconds({CPU_SAMPLE_N}, 1)[0] for _ in range({args.steps})]; "
            f"print(json.dumps(r))")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=3600)
    if out.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + out.stderr[-200:]}))
        return 0
    secs = json.loads(out.stdout.strip().splitlines()[-1])
    total = sum(secs)
    value = args.steps / total * (CPU_SAMPLE_N / n_full)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: grid 1250x1000 minus 20% gaps, n=1,000,000, Matern-1.5 rho=0.02, "
                               f"m=20, Poisson offset 1.0; each step a bounded sample at n={CPU_SAMPLE_N} "
                               f"scaled by n_sample/n"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"the CPU oracle (float64, sparse-LU Laplace) on the same recipe at "
                                   f"n={CPU_SAMPLE_N}, single thread, scaled linearly to n=1,000,000"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    legs = ws == 1 and rank == 0
    batch_problems = pregenerate("batched", args.batch) if legs and args.batch > 0 else None
    serve_arrivals = serve_problems = None
    if legs and args.serve_seconds > 0:
        import workloads as wl
        serve_arrivals = wl.poisson_arrivals(args.serve_rate, args.serve_seconds)
        serve_problems = pregenerate("serving", len(serve_arrivals))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = local
    torch.cuda.set_device(dev)
    import paper_2310_12000_gb300 as vl
    import workloads as wl

    P = wl.make_problem(WORKLOAD, seed=1 + rank, n=args.n)
    n = P.n
    ws_bytes = int(args.ws_gb * (1 << 30)) if args.ws_gb else int(min(torch.cuda.mem_get_info(dev)[0] * 0.6, 120 << 30))
    ctx = vl.Context(dev, ws_bytes=ws_bytes)
    stream = torch.cuda.current_stream(dev)
    pre = dict(precond=vl.PREC_LRAC, k=args.k) if args.precond == "lrac" else dict(precond=vl.PREC_VADU)
    pre["newton_eta_max"] = args.newton_eta_max
    o32 = vl.Opts.make(precision=vl.FP32_REFINE, t=50, cg_tol=1e-6, newton_tol=1e-7, cg_max_iter=3000, **pre)
    o64 = vl.Opts.make(precision=vl.FP64, t=50, cg_tol=1e-6, newton_tol=1e-7, cg_max_iter=3000, **pre)

    # neighbours + levels + factor, once per location set
    t0 = time.perf_counter()
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, o32)
    torch.cuda.synchronize(dev)
    graph_ms = 1000 * (time.perf_counter() - t0)
    info = fac.info()

    y_d = torch.from_numpy(P.y).to(f"cuda:{dev}")
    F_d = torch.from_numpy(P.F).to(f"cuda:{dev}")
    mode_d = torch.empty(n, dtype=torch.float64, device=f"cuda:{dev}")
    y_h = torch.from_numpy(P.y).pin_memory()
    F_h = torch.from_numpy(P.F).pin_memory()
    mode_h = torch.empty(n, dtype=torch.float64).pin_memory()

    def step(opts, host=False):
        fac.refit(P.sigma2, P.rho, opts)
        if host:
            st = fac.find_mode(P.lik, y_h.numpy(), F_h.numpy(), opts, mode_out=mode_h.numpy())
        else:
            st = fac.find_mode(P.lik, y_d, F_d, opts, mode_out=mode_d)
        L, ls = st.log_marglik(opts, with_stats=True)
        ls = dict(ls, mode=st.mode_stats())
        st.close()
        return L, ls

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x: float) -> float:
        return replica_throughput(x, 1)[0]

    for _ in range(args.warmup):
        step(o32)

    # ---------------- timed: device-resident inputs, kernel profiling on
    launches_before = ctx.profile_read("all")[1]
    ctx.profile(True)
    ctx.profile_read("all", reset=True)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lmls, stats = [], []
    with ClockSampler(dev) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            L, s = step(o32)
            lmls.append(L)
            stats.append(s)
        e1.record(stream)
        barrier()
    elapsed_s, value = replica_throughput(e0.elapsed_time(e1) / 1000.0, args.steps)
    launches = ctx.profile_read("all")[1]
    classes = ["sptrsv_fwd", "sptrsv_bwd", "spmv_B", "spmv_Bt", "coldot", "pcg_update", "factor", "woodbury",
               "slq_quad"]
    prof = {}
    for cls in classes:
        for t in (1, 50):
            ms, cnt = ctx.profile_read(cls, t)
            if cnt:
                prof[f"{cls}/t={t}"] = {"ms": ms, "launches": cnt}
        if cls == "factor":
            ms, cnt = ctx.profile_read(cls, 0)
            if cnt:
                prof["factor"] = {"ms": ms, "launches": cnt}
    ctx.profile(False)

    for cls in ("pivoted_cholesky", "lrac_gram", "lrac_kxk"):
        ms, cnt = ctx.profile_read(cls, args.k)
        if cnt:
            prof[cls] = {"ms": ms, "launches": cnt}

    # roofline for the dominant HBM-bound kernel class
    hbm_peak, peak_kind = _peaks()
    dom_key = max((k for k in prof if k.split("/")[0] in ("sptrsv_fwd", "sptrsv_bwd", "spmv_B", "spmv_Bt", "coldot",
                                                          "woodbury")),
                  key=lambda k: prof[k]["ms"])
    dcls, dt = dom_key.split("/")[0], int(dom_key.split("=")[1])
    avg_ms = prof[dom_key]["ms"] / prof[dom_key]["launches"]
    bytes_launch = algorithmic_bytes(dcls, n, P.m, dt, 4, args.k)
    achieved = bytes_launch / (avg_ms / 1000.0) / 1e9
    total_prof_ms = sum(v["ms"] for v in prof.values())
    roofline = {"bound": "hbm", "kernel": dom_key, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "traffic": _traffic(dcls, dt), "algorithmic_bytes_per_launch": bytes_launch,
                "avg_launch_ms": avg_ms,
                "share_of_profiled_time": prof[dom_key]["ms"] / total_prof_ms if total_prof_ms else None}

    # ---------------- e2e: host buffers, copies inside the timed region
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(2, min(args.steps, 3))
    for _ in range(e2e_steps):
        step(o32, host=True)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": ws * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * n * 8,
           "d2h_bytes_per_step": n * 8 + 8}

    # ---------------- FP64 reference on the GPU (the "vs FP64" part of the metric)
    fp64 = None
    if not args.no_fp64:
        barrier()
        t0 = time.perf_counter()
        L64, s64 = step(o64)
        barrier()
        fp64 = {"evals_per_s": ws / max_over_ranks(time.perf_counter() - t0), "lml": L64,
                "rel_diff_mixed_vs_fp64": abs(lmls[-1] - L64) / abs(L64),
                "newton": newton_summary(s64["mode"]), "slq_cg_iters_max": s64.get("cg_iters_max")}

    # ---------------- the config's second run: the low-rank preconditioner (rank k) on the same step
    lrac = None
    if args.precond != "lrac" and args.lrac_k > 0:
        olr = vl.Opts.make(precision=vl.FP32_REFINE, t=50, cg_tol=1e-6, newton_tol=1e-7, cg_max_iter=3000,
                           precond=vl.PREC_LRAC, k=args.lrac_k, newton_eta_max=args.newton_eta_max)
        barrier()
        ctx.profile(True)
        ctx.profile_read("all", reset=True)
        t0 = time.perf_counter()
        Llr, slr = step(olr)
        barrier()
        sec = max_over_ranks(time.perf_counter() - t0)
        lprof = {}
        for cls, tt in (("woodbury", 1), ("woodbury", 50), ("pivoted_cholesky", args.lrac_k),
                        ("lrac_gram", args.lrac_k), ("lrac_kxk", args.lrac_k)):
            ms, cnt = ctx.profile_read(cls, tt)
            if cnt:
                lprof[f"{cls}/t={tt}"] = {"ms": ms, "launches": cnt}
        ctx.profile(False)
        wb = lprof.get("woodbury/t=50")
        wroof = None
        if wb:
            byt = algorithmic_bytes("woodbury", n, P.m, 50, 4, args.lrac_k)
            ach = byt / (wb["ms"] / wb["launches"] / 1000.0) / 1e9
            wroof = {"bound": "hbm", "kernel": "woodbury/t=50 (two tcgen05 rank-k products + k x k)",
                     "achieved": ach, "peak": _peaks()[0], "unit": "GB/s", "frac": ach / _peaks()[0],
                     "algorithmic_bytes_per_launch": byt, "avg_launch_ms": wb["ms"] / wb["launches"]}
        lrac = {"k": args.lrac_k, "evals_per_s": ws / sec, "seconds_per_eval": sec, "lml": Llr,
                "rel_diff_vs_vadu": abs(Llr - lmls[-1]) / abs(lmls[-1]), "slq_stderr": slr.get("slq_stderr"),
                "newton": newton_summary(slr["mode"]), "slq_cg_iters_max": slr.get("cg_iters_max"),
                "probe_relres_max": slr.get("probe_relres_max"), "kernel_profile_ms": lprof,
                "woodbury_roofline": wroof,
                "note": "one evaluation (the pivoted Cholesky of Sigma is built in it: the factor is refit first)"}

    # ---------------- batched and serving legs (their own slot contexts)
    tune = vl.tune_report()
    ctx.close()
    del ctx, fac
    torch.cuda.empty_cache()
    batched = serving_out = None
    if batch_problems:
        from paper_2310_12000_gb300 import batched as bt
        batched = bt.run_merged(vl, batch_problems, device=dev, steps=2, warmup=1)
        batched.pop("lml", None)
        print(f"[bench] batched (merged): {batched['problems']} problems, {batched['seconds_per_batch']:.2f} s per "
              f"batch", file=sys.stderr, flush=True)
        if args.batch_streams:
            streams = bt.run_batch(vl, batch_problems, slots=args.slots, device=dev)
            streams.pop("lml", None)
            batched["streams"] = streams
        batched["workload"] = (f"{len(batch_problems)} problems, n log-uniform in [5e3, 5e4] (total "
                               f"{sum(p.n for p in batch_problems)}), m in {{10,20,30}}, uniform locations, "
                               f"exponential range U[0.02, 0.2], Bernoulli-logit, factor rows + mode + L^VLA (t=50), "
                               f"float32 + float64 refinement, merged into one block-diagonal system")
    if serve_problems:
        serving_out = serving_leg(vl, serve_problems, serve_arrivals, args.serve_seconds, args.slots, dev,
                                  args.small_slots, args.serve_form, args.group_slots, args.group_gb)
        print(f"[bench] serving: {serving_out['completed']} requests, p99 {serving_out['p99_latency_ms']} ms, "
              f"wall {serving_out['wall_s']:.1f} s", file=sys.stderr, flush=True)

    out = None
    if rank == 0:
        cb = cpu_baseline(n) if (ws == 1 and not args.no_cpu) else None
        s_last = stats[-1]
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * elapsed_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: " + ("1250x1000 grid" if args.n is None else "square grid")
                                   + f" on [0,1]^2 minus 20% rectangular gaps, "
                                   f"n={n}, Matern-1.5 sigma2=1 rho=0.02, m=20, Poisson-log offset 1.0, "
                                   f"t=50 Rademacher probes, "
                                   + (f"LRAC k={args.k}" if args.precond == "lrac" else "VADU")
                                   + ", float32 Krylov + float64 refinement, cg_tol 1e-6",
                       "step": "factor rows + Newton mode + SLQ log-marglik (neighbours/levels once, excluded)",
                       "l2": "inputs larger than L2 (probe block 1e6 x 56 float32 = 224 MB per vector)",
                       "graph_ms": graph_ms, "levels_fwd": info["nlev_fwd"], "levels_bwd": info["nlev_bwd"]},
            "lml": lmls[-1], "newton": newton_summary(s_last["mode"]),
            "slq_cg_iters_max": s_last.get("cg_iters_max"), "slq_cg_iters_total": s_last.get("cg_iters_total"),
            "slq_stderr": s_last.get("slq_stderr"), "probe_relres_max": s_last.get("probe_relres_max"),
            "probe_refine_steps": s_last.get("probe_refine_steps"),
            "fp64": fp64, "e2e": e2e, "gpu_launches": launches, "launches_before_timed": launches_before,
            "roofline": roofline,
            "kernel_profile_ms": prof, "clocks": clk.summary(), "cpu_baseline": cb,
            "p99_latency_ms": serving_out["p99_latency_ms"] if serving_out else None,
            "batched": batched, "serving": serving_out, "lrac": lrac, "launch_tuner": tune,
        }
        try:
            out.update(derived_metrics(prof, n, P.m, out["ms_per_step"], graph_ms))
        except Exception as exc:          # derived figures never cost the measured line
            out["derived_error"] = repr(exc)[:200]
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--n", type=int, default=None,
                    help="smaller instance of the same grid-with-gaps recipe (default: the 1,000,000-point grid)")
    ap.add_argument("--ws-gb", type=float, default=None, help="workspace size in GiB (default: 60%% of free memory)")
    ap.add_argument("--precond", default="vadu", choices=["vadu", "lrac"], help="preconditioner of the timed step")
    ap.add_argument("--k", type=int, default=500, help="LRAC rank")
    ap.add_argument("--lrac-k", type=int, default=500,
                    help="rank of the extra low-rank-preconditioner evaluation (0: skip it)")
    ap.add_argument("--newton-eta-max", type=float, default=0.1,
                    help="largest inexact-Newton forcing term (0: every Newton solve to cg_tol)")
    ap.add_argument("--batch", type=int, default=256, help="problems in the batched leg (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="arrival window of the serving leg (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=50.0, help="serving arrivals per second")
    ap.add_argument("--slots", type=int, default=16, help="slot contexts of the batched and serving legs")
    ap.add_argument("--batch-streams", action="store_true",
                    help="also run the batched problems on slot contexts (one stream each)")
    ap.add_argument("--serve-form", default="slots", choices=["groups", "slots"],
                    help="serving by one request per slot context, or by merged groups (continuous batching)")
    ap.add_argument("--group-slots", type=int, default=2, help="slot contexts of the merged-group serving form")
    ap.add_argument("--group-gb", type=float, default=60.0, help="workspace GiB of each merged-group slot")
    ap.add_argument("--small-slots", type=int, default=0,
                    help="of the serving slots, how many are sized for n <= 6e4 only (the rest for n = 2e5)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
