"""Benchmark of the GB300 inexact IETI-DP solver (MG-MG variant).

Workload: 2D Poisson on the quarter annulus (radii 1 and 2, exact NURBS map)
split into 6x6 patches, p = 3, 64x64 elements per patch (148,225 free dofs,
161,604 torn dofs, 3,900 multipliers, 85 primal dofs), vertex and
edge-average primal constraints, f from the manufactured solution
u = sin(pi x) sin(pi y) (r-1)(2-r).  Synthetic, deterministic input.

A step solves a batch of B (default 8) independent copies of the workload,
each with its own assembled problem and handle, in lockstep
(``ietidp_solve_batch``): for every copy d = B K~^{-1} f, the dual PCG to
1e-10 with the scaled Dirichlet preconditioner and the recovery of u, with
the local solves of all 36 x B patches merged into shared launches.  Load
vectors are resident in HBM; setup is timed separately.  The headline is the
mixed path (FP32 V-cycles under FP64 CG); the FP64 path is timed beside it,
and single solves (one copy at a time) give the latency.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (the solver has no
cross-GPU exchange step); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

# the oracle legs (cpu_baseline, --impl reference) report one host core: the
# BLAS / OpenMP pools are pinned to one thread before numpy loads them
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1705_04531_gb300 import workloads as W  # noqa: E402

WORKLOAD = "annulus6x6_p3_n64"
METRIC = "IETI-DP solves/sec (mixed FP32 V-cycles / FP64 CG, rel err <= 1e-8)"
UNIT = "solves/s"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--vcycle-reps", type=int, default=50)
    ap.add_argument("--mode", default="bench", choices=["bench", "vcycle", "serve", "profile", "phases"],
                    help="vcycle: setup plus three batched V-cycle launches (profiling target); "
                         "serve: Poisson-arrival request stream through the continuous-batching server; "
                         "profile: one batched solve of --batch copies inside a profiler range "
                         "(cudaProfilerStart/Stop), after a warm-up solve; "
                         "phases: per-phase times of a batched V-cycle (library built with "
                         "IETIDP_PHASE_TIMERS=1)")
    ap.add_argument("--sm-mhz", type=float, default=2070.0, help="phases: SM clock for cycle counts")
    ap.add_argument("--mg-kind", default="standard", choices=["standard", "highorder"],
                    help="phases: multigrid of the solvers")
    ap.add_argument("--rate", type=float, default=None, help="serve: arrivals per second (one rate)")
    ap.add_argument("--nreq", type=int, default=512, help="serve: requests in the stream")
    ap.add_argument("--concurrency", type=int, default=8, help="serve: worker streams")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="serve: device memory budget")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--method", default="dual", choices=["dual", "saddle", "dmg"],
                    help="serve / profile: outer method (MG-MG, MG-MG-S, D-MG)")
    ap.add_argument("--batch", type=int, default=8,
                    help="independent copies of the workload solved in lockstep per step")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads (2x2 square, uneven 8x8, 2x2x2 cube) and the serving stream")
    ap.add_argument("--serve-rates", default="100,1000", help="default run: arrival rates of the serving stream")
    a = ap.parse_args()
    a.rate_given = a.rate is not None
    return a


def workload(name):
    return W.by_name(name)


# ---------------------------------------------------------------------------
# algorithmic bytes of the batched Neumann solver kernel (per CG iteration of
# one patch): V-cycle at nu1 = nu2 = 2 + FP64 stiffness SpMV + CG vectors
# ---------------------------------------------------------------------------
def levels(nelem, degree, cmin=4):
    sched = [tuple(nelem)]
    while True:
        cur = sched[-1]
        nxt = tuple(n // 2 if (n > cmin and n % 2 == 0) else n for n in cur)
        if nxt == cur:
            break
        sched.append(nxt)
    sched = sched[::-1]
    out = []
    for ne in sched:
        n = int(np.prod([a + p for a, p in zip(ne, degree)]))
        S = int(np.prod([2 * p + 1 for p in degree]))
        out.append((n, S))
    return out


def bytes_per_iteration(nelem, degree, sv, nu=4):
    lv = levels(nelem, degree)
    b = 0
    for l in range(1, len(lv)):
        n, S = lv[l]
        nc = lv[l - 1][0]
        b += (nu + 1) * (S * n * sv + 3 * n * sv)       # sweeps + residual: values, x, b, x/r write
        b += 3 * n * sv + 2 * nc * sv                   # restriction and prolongation
    n0 = lv[0][0]
    b += n0 * n0 * sv + 2 * n0 * sv                     # coarsest dense solve
    n, S = lv[-1]
    b += S * n * 8 + 2 * n * 8                          # FP64 SpMV q = K p
    b += 12 * n * 8 + n * (8 + sv) * 2                  # CG vector updates, dots, casts
    return b


def vcycle_bytes(nelem, degree, sv, nu=4):
    lv = levels(nelem, degree)
    b = 0
    for l in range(1, len(lv)):
        n, S = lv[l]
        nc = lv[l - 1][0]
        b += (nu + 1) * (S * n * sv + 3 * n * sv) + 3 * n * sv + 2 * nc * sv
    n0 = lv[0][0]
    return b + n0 * n0 * sv + 2 * n0 * sv


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def oracle_run(dom, budget_s=60.0, min_solves=20):
    """The oracle (D-D variant: sparse LU local solves) timed on one host core
    on complete solves of the same workload (setup excluded): `min_solves`
    solves or `budget_s` seconds, whichever comes first."""
    from oracle import ietidp as O
    t0 = time.perf_counter()
    s = O.IETIDP(dom, O.Options(mode="direct"))
    t_setup = time.perf_counter() - t0
    times = []
    u = None
    while True:
        s.stats = O.Stats()
        t = time.perf_counter()
        u = s.solve()
        times.append(time.perf_counter() - t)
        if sum(times) > budget_s or len(times) >= min_solves:
            break
    return {"u": u, "times": times, "setup_s": t_setup, "outer_it": s.stats.outer_it}


def _oracle_worker(job):
    """Child process of the multi-core oracle legs: set-up, then `n` timed
    solves in the given mode (one core per process)."""
    mode, n, name = job
    from oracle import ietidp as O
    s = O.IETIDP(workload(name), O.Options(mode=mode))
    times = []
    for _ in range(n):
        s.stats = O.Stats()
        t = time.perf_counter()
        s.solve()
        times.append(time.perf_counter() - t)
    return times


def oracle_legs(name):
    """The oracle beside its D-D 1-core figure: the MG-MG mode (multigrid
    local solves) on one core, one complete solve; the D-D mode on every host
    core, one process per core solving its own copy (spawned processes, so no
    CUDA state is inherited)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    ncores = os.cpu_count() or 1
    out = {}
    with ctx.Pool(1) as pool:
        t = pool.map(_oracle_worker, [("mg", 1, name)])[0]
    out["mg_1core"] = {"value": len(t) / sum(t), "unit": UNIT, "cores": 1, "solves": len(t),
                       "sample": f"{len(t)} complete MG-MG solve of {name} (multigrid local solves), setup excluded"}
    with ctx.Pool(ncores) as pool:
        res = pool.map(_oracle_worker, [("direct", 2, name)] * ncores)
    wall = max(sum(r) for r in res)
    nsol = sum(len(r) for r in res)
    out["dd_all_cores"] = {"value": nsol / wall, "unit": UNIT, "cores": ncores, "solves": nsol,
                           "sample": f"{ncores} processes x 2 complete D-D solves of {name}, setup excluded; "
                                     f"time = the slowest process's solve time"}
    return out


def relerr(got, ref):
    return float(np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(got, ref)) /
                         sum(np.sum(b ** 2) for b in ref)))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    dom = workload(args.workload)
    from oracle import ietidp as O
    s = O.IETIDP(dom, O.Options(mode="direct"))
    for _ in range(max(0, min(args.warmup, 1))):
        s.stats = O.Stats()
        s.solve()
    times = []
    for _ in range(args.steps):
        s.stats = O.Stats()
        t = time.perf_counter()
        s.solve()
        times.append(time.perf_counter() - t)
    v = len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "variant": "D-D (CPU oracle)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} complete solves of {args.workload}, setup excluded"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x, dist, device):
    """Largest value of x over the ranks (x itself without a process group)."""
    if not dist:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(max_ms, world, batch, steps):
    """Whole-job throughput: every rank solves `batch` copies per step (weak
    scaling, independent replicas); time = the slowest rank's."""
    return world * batch * steps / (max_ms / 1e3)


def time_path(api, torch, prob, prec, args, flush, stream):
    t0 = time.perf_counter()
    sol = api.Solver(prob, precision=prec)
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t0)
    f = prob.load()
    u = torch.empty(sol.n_torn, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        sol.solve(f, u)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        _, st = sol.solve(f, u)
        ev[k][1].record(stream)
        stats.append(st)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    return sol, u, ms, stats, setup_ms


def time_batch(api, torch, dom, prec, args, flush, stream, method="dual"):
    """B independent copies of the workload (own assembled problem and handle
    each) solved in lockstep by ietidp_solve_batch: one step = B complete
    solves, their local solves merged into shared launches.  Timed with CUDA
    events on the launching stream."""
    B = args.batch
    t0 = time.perf_counter()
    probs = [api.Problem(dom) for _ in range(B)]
    sols = [api.Solver(p, precision=prec, method=method) for p in probs]
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t0) / B
    fs = [p.load() for p in probs]
    us = [torch.empty(s.n_torn, dtype=torch.float64, device="cuda") for s in sols]
    for _ in range(args.warmup):
        api.Solver.solve_batch(sols, fs, us)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    n0 = api.kernel_launches()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        _, st = api.Solver.solve_batch(sols, fs, us)
        ev[k][1].record(stream)
        stats.append(st)
    torch.cuda.synchronize()
    launches = api.kernel_launches() - n0
    ms = [a.elapsed_time(b) for a, b in ev]
    return {"sols": sols, "probs": probs, "fs": fs, "us": us, "ms": ms, "stats": stats,
            "launches": launches, "setup_ms": setup_ms}


def time_copies(api, torch, dom, prec, B, steps, warmup, flush, stream, method="dual"):
    """B independent copies of `dom` solved in lockstep (ietidp_solve_batch);
    CUDA events on the launching stream around each of `steps` timed steps."""
    t0 = time.perf_counter()
    probs = [api.Problem(dom) for _ in range(B)]
    sols = [api.Solver(p, precision=prec, method=method) for p in probs]
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t0) / B
    fs = [p.load() for p in probs]
    us = [torch.empty(s.n_torn, dtype=torch.float64, device="cuda") for s in sols]
    for _ in range(warmup):
        api.Solver.solve_batch(sols, fs, us)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stats = []
    n0 = api.kernel_launches()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        _, st = api.Solver.solve_batch(sols, fs, us)
        ev[k][1].record(stream)
        stats.append(st)
    torch.cuda.synchronize()
    launches = api.kernel_launches() - n0
    ms = [a.elapsed_time(b) for a, b in ev]
    return {"sols": sols, "probs": probs, "fs": fs, "us": us, "ms": ms, "stats": stats,
            "launches": launches, "setup_ms": setup_ms}


def batched_vcycles(api, torch, bt, reps=10):
    """One V-cycle over the Neumann hierarchies of every patch of every copy
    in merged launches (ietidp_vcycles_batch): median duration of `reps`."""
    xs = [torch.zeros_like(f) for f in bt["fs"]]
    for _ in range(2):
        api.Solver.vcycles_batch(bt["sols"], bt["fs"], xs, 1)
    return float(np.median([api.Solver.vcycles_batch(bt["sols"], bt["fs"], xs, 1) for _ in range(reps)]))


def patch_avg_bytes(dom, sv):
    """Algorithmic bytes of one CG iteration averaged over the patches."""
    return float(np.mean([bytes_per_iteration(dom.patch_nelem(k), dom.patch_degree(k), sv)
                          for k in range(dom.npatch)]))


def extra_workload(api, torch, name, B, steps, warmup, flush, stream, peak):
    """Solves/s, latency, iterations, accuracy against the FP64 path, batched
    V-cycle DoF/s and the merged Neumann launches against the HBM roofline for
    one more workload (mixed path, B copies per step; one copy for latency)."""
    dom = workload(name)
    bt = time_copies(api, torch, dom, "mixed", B, steps, warmup, flush, stream)
    sts = bt["stats"]
    ms = bt["ms"]
    s0, f0, u0 = bt["sols"][0], bt["fs"][0], bt["us"][0]
    lat = []
    for k in range(steps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        s0.solve(f0, u0)
        e1.record(stream)
        torch.cuda.synchronize()
        if k > 0:
            lat.append(e0.elapsed_time(e1))
    ref_sol = api.Solver(bt["probs"][0], precision="fp64")
    uref, st64 = ref_sol.solve(f0)
    torch.cuda.synchronize()
    uref_p = ref_sol.split(uref)
    err = max(relerr(bt["sols"][i].split(bt["us"][i]), uref_p) for i in range(B))
    ref_sol.close()
    vc_ms = batched_vcycles(api, torch, bt)
    nfine = sum(dom.patch_ndof(k) for k in range(dom.npatch)) * B
    bpi = patch_avg_bytes(dom, 4)
    iters = sum(s["inner_its"] for st in sts for s in st)
    nl = sum(st[0]["neumann_launches"] for st in sts)
    kms = sum(st[0]["neumann_ms"] for st in sts)
    alg = iters * bpi / max(1, nl)
    lms = kms / max(1, nl)
    ach = alg / (lms / 1e3) / 1e9
    out = {"value": B * len(ms) / (sum(ms) / 1e3), "unit": "solves/s", "batch": B,
           "ms_per_step": sum(ms) / len(ms),
           "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
           "single_p50_ms": float(np.percentile(lat, 50)), "single_p99_ms": float(np.percentile(lat, 99)),
           "outer_it": sts[-1][0]["outer_it"], "inner_it_avg": sts[-1][0]["inner_it_avg"],
           "outer_it_fp64": st64["outer_it"], "rel_err_vs_fp64_gpu": err,
           "setup_ms": bt["setup_ms"],
           "vcycle_dofs_per_s_batched": nfine / (vc_ms / 1e3), "vcycle_ms_batched": vc_ms,
           "roofline": {"bound": "hbm", "kernel": "merged Neumann PCG + V-cycle launches (all specialisations)",
                        "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "alg_bytes_per_launch": alg, "launch_ms": lms, "launches": nl,
                        "bytes_per_cg_iteration": "patch average (CG iterations taken equal across patches)"},
           "patches": dom.npatch, "torn_dofs": int(nfine // B)}
    close_batch(bt)
    return out


def highorder_compare(api, torch, flush, stream, steps=2):
    """The paper's high-degree settings (Sec. 4; p = 4 and 7 in Tables 1 and
    2): quarter annulus 6x6, n = 32, one solve at a time, with the high-order
    multigrid (degree 1 below the finest level, subspace-corrected mass
    smoother) and with the standard one (degree p on every level,
    Gauss-Seidel); accuracy against the FP64 high-order solve (the first
    run).  A set-up or solve that does not converge within the default
    iteration caps is reported as such."""
    out = {}
    # p = 7: one timed solve each, no warm-up (the standard multigrid takes
    # over a minute per solve); the mixed path is not run there (the FP32
    # storage of the degree-7 operator keeps the inner CG from its tolerance)
    plan = {4: ((("highorder", "fp64"), ("highorder", "mixed"), ("standard", "mixed")), steps, True),
            7: ((("highorder", "fp64"), ("standard", "mixed")), 1, False)}
    for p_ in (4, 7):
        runs, nsteps, warm = plan[p_]
        dom = W.annulus_6x6(32, p_)
        prob = api.Problem(dom)
        res = {"patches": dom.npatch, "degree": p_, "elements_per_patch": "32x32",
               "torn_dofs": int(sum(dom.patch_ndof(k) for k in range(dom.npatch)))}
        uref_p = None
        for kind, prec in runs:
            key = f"{kind}_{prec}"
            sol = None
            try:
                t0 = time.perf_counter()
                sol = api.Solver(prob, precision=prec, mg_kind=kind)
                torch.cuda.synchronize()
                setup_ms = 1e3 * (time.perf_counter() - t0)
                u = None
                if warm:
                    u, st = sol.solve()
                lat = []
                for _ in range(nsteps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    flush.zero_()
                    e0.record(stream)
                    u, st = sol.solve(None, u)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    lat.append(e0.elapsed_time(e1))
            except api.IetidpError as e:
                res[key] = {"failed": str(e)}
                if sol is not None:
                    sol.close()
                continue
            got = sol.split(u)
            if uref_p is None:
                uref_p = got
            res[key] = {"solves_per_s": 1e3 / float(np.median(lat)), "p50_ms": float(np.median(lat)),
                        "outer_it": st["outer_it"], "inner_it_avg": st["inner_it_avg"],
                        "converged": bool(st["converged"]),
                        "rel_err_vs_fp64_highorder": relerr(got, uref_p), "setup_ms": setup_ms}
            sol.close()
        prob.close()
        out[dom.name] = res
    return out


def serve_stream(api, torch, nreq, rate, seed, concurrency, budget_gb, precision="mixed", method="dual"):
    """Poisson-arrival request stream through the continuous-batching server:
    solves/s, p50/p99 latency (arrival to result) and the peak of the
    admitted requests' estimated device memory (sampled every 5 ms)."""
    reqs = W.serving_stream(nreq=nreq, rate=rate, seed=seed)
    srv = api.Server(int(budget_gb * (1 << 30)), max_concurrent=concurrency, precision=precision, method=method)
    srv.wait(srv.submit(W.serving_stream(nreq=1, rate=1.0, seed=99, ms=(2,), ns=(16,))[0].domain))
    torch.cuda.synchronize()
    peak = [0]
    stop = threading.Event()

    def sample():
        while not stop.is_set():
            try:
                peak[0] = max(peak[0], srv.status()["in_flight_bytes"])
            except Exception:
                pass
            time.sleep(0.005)

    th = threading.Thread(target=sample, daemon=True)
    th.start()
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        dt = t0 + r.arrival - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets.append(srv.submit(r.domain))
    lat, runs, its = [], [], []
    for t in tickets:
        state, u, st, tm = srv.wait(t)
        lat.append(tm["latency_s"])
        runs.append(tm["run_s"])
        its.append(st["outer_it"])
    t1 = time.perf_counter()
    stop.set()
    th.join(timeout=1.0)
    srv.close()
    return {"rate_per_s": rate, "requests": nreq, "seed": seed, "value": nreq / (t1 - t0), "unit": "solves/s",
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "run_p50_ms": 1e3 * float(np.percentile(runs, 50)), "outer_it_mean": float(np.mean(its)),
            "admitted_bytes_peak": int(peak[0]), "wall_s": t1 - t0}


def close_batch(bt):
    for s in bt["sols"]:
        s.close()
    for p in bt["probs"]:
        p.close()


def roofline(bt, dom, sv):
    """Dominant kernel: the merged local Neumann solve launch (all patches of
    all B handles).  Algorithmic bytes per launch = CG iterations of all its
    slots x bytes per iteration; duration from the engine's CUDA events."""
    p = dom.patch_degree(0)
    ne = dom.patch_nelem(0)
    bpi = bytes_per_iteration(ne, p, sv)
    iters = sum(s["inner_its"] for st in bt["stats"] for s in st)
    nlaunch = sum(st[0]["neumann_launches"] for st in bt["stats"])
    kms = sum(st[0]["neumann_ms"] for st in bt["stats"])
    alg = iters * bpi / max(1, nlaunch)
    launch_ms = kms / max(1, nlaunch)
    achieved = alg / (launch_ms / 1e3) / 1e9
    return achieved, alg, launch_ms, nlaunch


def run_vcycle_probe(args):
    """Setup of the workload and three batched V-cycle launches over the
    Neumann hierarchies of all patches (a short, self-contained profiling
    target for the dominant kernel)."""
    import torch
    from paper_1705_04531_gb300 import build
    build.build()
    from paper_1705_04531_gb300 import ietidp as api
    dom = workload(args.workload)
    prob = api.Problem(dom)
    sol = api.Solver(prob, precision=args.precision)
    f = prob.load()
    x = torch.zeros_like(f)
    for _ in range(3):
        sol.vcycles(f, x, 1)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "vcycle", "workload": args.workload, "precision": args.precision,
                      "x_norm": float(x.norm())}))


def run_phases(args):
    """Phase breakdown of one batched V-cycle (--batch copies of the
    workload, Neumann hierarchies of every patch, plus the fine operator of
    the CG) from the in-kernel clock counters of CTA 0 (a library built with
    IETIDP_PHASE_TIMERS=1; all zero otherwise): microseconds per V-cycle at
    the SM clock given by --sm-mhz, averaged over ten launches."""
    import torch
    from paper_1705_04531_gb300 import build
    build.build()
    from paper_1705_04531_gb300 import ietidp as api
    dom = workload(args.workload)
    probs = [api.Problem(dom) for _ in range(args.batch)]
    sols = [api.Solver(p_, precision=args.precision, mg_kind=args.mg_kind) for p_ in probs]
    api.Solver.solve_batch(sols)        # autotuning of the merged launches
    fs = [p_.load() for p_ in probs]
    xs = [torch.zeros_like(f) for f in fs]
    for _ in range(2):
        api.Solver.vcycles_batch(sols, fs, xs, 1)
    q0 = sols[0].phase_timers()
    ms = [api.Solver.vcycles_batch(sols, fs, xs, 1) for _ in range(10)]
    q1 = sols[0].phase_timers()
    dq = (q1 - q0) / 10 / args.sm_mhz
    names = {48: "coarsest", 49: "fine_operator", 52: "ho_fine_residuals", 53: "ho_smoother",
             54: "ho_restriction", 55: "ho_degree1_vcycle", 56: "ho_prolongation",
             57: "generic_fine_operator", 58: "generic_conversions"}
    for l in range(1, 12):
        for k, nm in enumerate(["sweeps", "residual", "restrict", "prolong"]):
            names[4 * l + k] = f"level{l}_{nm}"
    print(json.dumps({"mode": "phases", "workload": args.workload, "batch": args.batch,
                      "precision": args.precision, "mg_kind": args.mg_kind, "launch_ms": float(np.median(ms)),
                      "phase_us": {names[i]: round(float(dq[i]), 1) for i in sorted(names) if dq[i] != 0}}))


def run_serve(args):
    """Serving stream (m x m unit-square patch grids, m in {2,4,6,8}, p in
    {2,3}, 16..128 elements per patch direction, f = 8 random sine modes,
    Poisson arrivals) through the continuous-batching server, one line per
    rate of --serve-rates (or --rate when given)."""
    import torch
    from paper_1705_04531_gb300 import build
    build.build()
    from paper_1705_04531_gb300 import ietidp as api
    rates = [args.rate] if args.rate_given else [float(v) for v in args.serve_rates.split(",") if v]
    for r in rates:
        res = serve_stream(api, torch, args.nreq, r, 0, args.concurrency, args.budget_gb, args.precision, args.method)
        res.update({"mode": "serve", "metric": "IETI-DP solves/sec (serving stream, each request assembled, "
                                              "set up and solved)", "n_gpus": 1,
                    "config": {"concurrency": args.concurrency, "budget_gb": args.budget_gb,
                               "precision": args.precision, "method": args.method}})
        print(json.dumps(res), flush=True)


def run_profile(args):
    """A warm-up batched solve (autotuning included), then one batched solve
    of --batch copies of the workload inside a profiler range, so that
    ``ncu --profile-from-start off -k regex:k_solve_t -c 1`` captures the
    first merged local-solve launch of a tuned, steady-state solve."""
    import torch
    from paper_1705_04531_gb300 import build
    build.build()
    from paper_1705_04531_gb300 import ietidp as api
    dom = workload(args.workload)
    probs = [api.Problem(dom) for _ in range(args.batch)]
    sols = [api.Solver(p, precision=args.precision, method=args.method) for p in probs]
    api.Solver.solve_batch(sols)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    _, sts = api.Solver.solve_batch(sols)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    p, ne = dom.patch_degree(0), dom.patch_nelem(0)
    its = sum(st["inner_its"] for st in sts)
    nl = sts[0]["neumann_launches"]
    print(json.dumps({"mode": "profile", "workload": args.workload, "batch": args.batch,
                      "precision": args.precision, "method": args.method, "outer_it": sts[0]["outer_it"],
                      "neumann_launches": nl,
                      "cg_iterations_per_launch": its / max(1, nl),
                      "alg_bytes_per_cg_iteration": bytes_per_iteration(ne, p, 4 if args.precision == "mixed" else 8),
                      "autotune": api.autotune_table()}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "vcycle":
        return run_vcycle_probe(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "profile":
        return run_profile(args)
    if args.mode == "phases":
        return run_phases(args)
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1705_04531_gb300 import build
    build.build()
    from paper_1705_04531_gb300 import ietidp as api

    dom = workload(args.workload)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    prob = api.Problem(dom)
    torch.cuda.synchronize()
    assemble_ms = 1e3 * (time.perf_counter() - t0)

    # single solves (latency): FP64 path, then the mixed path
    sol64, u64, ms64, st64, setup64 = time_path(api, torch, prob, "fp64", args, flush, stream)
    u64h = sol64.split(u64)
    sol64.close()
    sol, u, ms1, sts1, setup_ms = time_path(api, torch, prob, "mixed", args, flush, stream)
    uh = sol.split(u)

    # V-cycle throughput: one batched V-cycle over all 36 Neumann hierarchies per launch
    f = prob.load()
    x = torch.zeros_like(f)
    for _ in range(3):
        sol.vcycles(f, x, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.vcycle_reps):
        sol.vcycles(f, x, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    vc_ms = e0.elapsed_time(e1) / args.vcycle_reps
    nfine = sum(dom.patch_ndof(k) for k in range(dom.npatch))
    vcycle_dofs_s = nfine / (vc_ms / 1e3)
    n_torn, n_lambda, n_primal = sol.n_torn, sol.info.n_lambda, sol.info.n_primal
    sol.close()
    del x, f

    # batched FP64 path (comparison), then the batched mixed path (headline)
    bt64 = time_batch(api, torch, dom, "fp64", args, flush, stream)
    b64_err = max(relerr(bt64["sols"][i].split(bt64["us"][i]), u64h) for i in range(args.batch))
    # every whole-job figure takes the slowest rank's time (all ranks call these)
    ms64b = max_over_ranks(sum(bt64["ms"]), dist, "cuda")
    ms64s = max_over_ranks(sum(ms64), dist, "cuda")
    ms1s = max_over_ranks(sum(ms1), dist, "cuda")
    ach64, _, lms64, _ = roofline(bt64, dom, 8)
    close_batch(bt64)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        bt = time_batch(api, torch, dom, "mixed", args, flush, stream)
    ms = bt["ms"]
    tot = max_over_ranks(sum(ms), dist, "cuda")
    value = job_value(tot, world, args.batch, args.steps)
    ub = [bt["sols"][i].split(bt["us"][i]) for i in range(args.batch)]

    # e2e through the C ABI with host buffers (pinned), copies inside the timed region
    fhs, uhs = [], []
    for i in range(args.batch):
        fh = torch.empty(n_torn, dtype=torch.float64).pin_memory()
        fh.copy_(bt["fs"][i].cpu())
        fhs.append(fh)
        uhs.append(torch.empty(n_torn, dtype=torch.float64).pin_memory())
    fnp, unp = [t_.numpy() for t_ in fhs], [t_.numpy() for t_ in uhs]
    api.Solver.solve_batch_host(bt["sols"], fnp, unp)
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        api.Solver.solve_batch_host(bt["sols"], fnp, unp)
        e2e_t.append(time.perf_counter() - t)
    e2e_val = world * args.batch * len(e2e_t) / max_over_ranks(sum(e2e_t), dist, "cuda")
    achieved, alg_bytes_per_launch, launch_ms, nlaunch = roofline(bt, dom, 4)
    sts = bt["stats"]
    bvc_ms = batched_vcycles(api, torch, bt)
    bvc_dofs = nfine * args.batch / (bvc_ms / 1e3)
    close_batch(bt)

    # MG-MG-S (BPCG on the saddle-point system, 3 V-cycles in the K~
    # preconditioner), batched mixed path on the same workload
    bs = time_batch(api, torch, dom, "mixed", args, flush, stream, method="saddle")
    saddle_err = max(relerr(bs["sols"][i].split(bs["us"][i]), u64h) for i in range(args.batch))
    ms_s = max_over_ranks(sum(bs["ms"]), dist, "cuda")
    saddle = {"value": job_value(ms_s, world, args.batch, args.steps),
              "ms_per_step": ms_s / args.steps,
              "outer_it": bs["stats"][-1][0]["outer_it"], "vcycles_per_solve": bs["stats"][-1][0]["vcycles"],
              "rel_err_vs_fp64_dual": saddle_err,
              "note": "MG-MG-S: Bramble-Pasciak CG on Eq. 2, mixed V-cycles, same batch and tolerance"}
    close_batch(bs)

    # D-MG (direct banded Cholesky Neumann solves, multigrid Dirichlet
    # problems), batched mixed path on the same workload
    bd = time_batch(api, torch, dom, "mixed", args, flush, stream, method="dmg")
    dmg_err = max(relerr(bd["sols"][i].split(bd["us"][i]), u64h) for i in range(args.batch))
    ms_d = max_over_ranks(sum(bd["ms"]), dist, "cuda")
    dmg = {"value": job_value(ms_d, world, args.batch, args.steps),
           "ms_per_step": ms_d / args.steps,
           "outer_it": bd["stats"][-1][0]["outer_it"], "setup_ms": bd["setup_ms"],
           "rel_err_vs_fp64_dual": dmg_err,
           "note": "D-MG: direct banded-Cholesky local Neumann solves, multigrid Dirichlet problems, same batch"}
    close_batch(bd)
    peak, peak_kind = peaks()
    # the other workloads of the benchmark family and the serving stream
    # (single process only: with several ranks the line reports the headline)
    extra, serve, highorder = {}, [], None
    if world == 1 and not args.no_extra:
        xs_ = min(args.steps, 5)
        for nm, B in (("square2x2_p2_n16", 8), ("uneven8x8_s0", 2), ("cube2x2x2_p2_n32", 4)):
            extra[nm] = extra_workload(api, torch, nm, B, xs_, 2, flush, stream, peak)
        for r_ in [float(v) for v in args.serve_rates.split(",") if v]:
            serve.append(serve_stream(api, torch, args.nreq, r_, 0, args.concurrency, args.budget_gb))
        highorder = highorder_compare(api, torch, flush, stream)
    tune = api.autotune_table()

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.txt")
    if os.path.exists(tp):
        with open(tp) as fh_:
            for ln in fh_:
                f_ = ln.split()
                if len(f_) == 2 and not ln.startswith("#") and f_[0] == args.workload:
                    traffic = float(f_[1])

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot / args.steps,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycle + f64 CG",
        "data": "synthetic",
        "config": {"workload": args.workload, "patches": dom.npatch, "degree": 3, "elements_per_patch": "64x64",
                   "free_dofs": 148225, "torn_dofs": n_torn, "multipliers": n_lambda,
                   "primal": n_primal, "precision": "mixed", "tol_outer": 1e-10,
                   "l2": f"{L2_FLUSH_BYTES >> 20} MiB buffer written between timed steps; "
                         f"working set {args.batch} x ~110 MB > L2",
                   "replicas": world, "batch": args.batch,
                   "step": f"{args.batch} independent copies of the workload (own problem and handle each) "
                           f"solved in lockstep by ietidp_solve_batch",
                   "autotune": tune},
        "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
        "single": {"value": job_value(ms1s, world, 1, args.steps), "ms_per_step": ms1s / args.steps,
                   "p50_ms": float(np.percentile(ms1, 50)), "p99_ms": float(np.percentile(ms1, 99)),
                   "note": "one solve at a time (latency: 36 CTAs on 152 SMs)"},
        "outer_it": sts[-1][0]["outer_it"], "inner_it_avg": sts[-1][0]["inner_it_avg"],
        "kappa": sts[-1][0]["kappa"],
        "setup_ms": setup_ms, "assemble_ms": assemble_ms,
        "fp64": {"value": job_value(ms64b, world, args.batch, args.steps),
                 "ms_per_step": ms64b / args.steps,
                 "single_value": job_value(ms64s, world, 1, args.steps),
                 "single_p50_ms": float(np.percentile(ms64, 50)),
                 "outer_it": st64[-1]["outer_it"], "inner_it_avg": st64[-1]["inner_it_avg"],
                 "setup_ms": setup64, "batch_vs_single_rel_err": b64_err,
                 "roofline_achieved_gbs": ach64, "launch_ms": lms64},
        "mixed_over_fp64": ms64b / tot,
        "mg_mg_s": saddle,
        "d_mg": dmg,
        "vcycle_dofs_per_s": vcycle_dofs_s, "vcycle_ms": vc_ms,
        "vcycle_dofs_per_s_batched": bvc_dofs, "vcycle_ms_batched": bvc_ms,
        "roofline": {"bound": "hbm", "kernel": "k_solve_t<float,2,3,3,0> (merged Neumann PCG + V-cycles)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": traffic,
                     "alg_bytes_per_launch": alg_bytes_per_launch,
                     "launch_ms": launch_ms, "launches": nlaunch},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 8 * n_torn * args.batch,
                "d2h_bytes_per_step": 8 * n_torn * args.batch},
        "gpu_launches": int(bt["launches"]),
        "clocks": clk.summary(),
    }
    if extra:
        line["workloads"] = extra
    if highorder:
        line["highorder"] = highorder
    if serve:
        line["serve"] = {"stream": f"{args.nreq} requests, m x m unit-square patches, m in {{2,4,6,8}}, p in {{2,3}}, "
                                   "n in {16,32,64,128}, f = 8 random sine modes, Poisson arrivals",
                         "concurrency": args.concurrency, "budget_gb": args.budget_gb, "rates": serve}
    if not args.no_cpu_baseline:
        orc = oracle_run(dom)
        ref = orc["u"]
        line["rel_err_mixed"] = max(relerr(x_, ref) for x_ in ub)
        line["rel_err_mixed_single"] = relerr(uh, ref)
        line["rel_err_fp64"] = relerr(u64h, ref)
        v = len(orc["times"]) / sum(orc["times"])
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{len(orc['times'])} complete D-D solves of {args.workload} "
                                          f"(sparse LU local solves), setup excluded",
                                "outer_it": orc["outer_it"], "p50_ms": 1e3 * float(np.percentile(orc["times"], 50)),
                                "p99_ms": 1e3 * float(np.percentile(orc["times"], 99))}
        line["cpu_baseline"].update(oracle_legs(args.workload))
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
