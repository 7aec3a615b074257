#!/usr/bin/env python
"""Throughput of the hierarchical solver on one GB300 (or N replicas).

Workload (one step): the 3D 7-point Poisson matrix on a 64^3 grid (n = 262144,
Dirichlet), leaf clusters of 64 unknowns by coordinate bisection (depth 12),
for each eps in {1e-2, 1e-4, 1e-6}: factor (Algorithm 1) and solve 16 seeded
uniform[-1,1] right-hand sides with GMRES(30) preconditioned by the factor to
relative residual 1e-10.  Metric: unknowns/s = len(eps) * n * nrhs / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lrs|reference]

After the timed region the same JSON line also reports the precision form
(block products on the tensor cores) on that workload, repeated-solve
latencies, the batched form (seeded 2D upwind convection-diffusion instances,
side U[64, 512], factored 64 at a time through lrs_analyze_batch and solved by
per-instance GMRES; all 256 instances as four groups) and the serving form under a seeded Poisson-arrival request stream.  The
CPU baseline (the FP64 oracle, one core, on the full 64^3 matrix at the
sweep's first eps) runs in a separate process started before any GPU work and
overlaps the GPU measurements.

Prints one JSON line (rank 0).  `value` is timed with CUDA events on the
library's stream with inputs resident in HBM; `e2e` repeats the step through
the C ABI with pinned host buffers (copies inside the timed region).  Under
torchrun every rank runs its own replica of the workload (no data-path
collective); the slowest rank's time sets the whole-job value.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "unknowns/s factor+GMRES to rel-res 1e-10 vs plain FP64; p50/p99 solve latency"
FP64_PEAK_GFLOPS = 1250.0   # 152 SMs x 2 FP64 FMA/clk x 2 flop x ~2.06 GHz (nominal 1.25 TFLOP/s)
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.06   # 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.06 GHz
# DRAM bytes (read + write) per algorithmic byte of the FP64 gather GEMM, from
# one ncu capture of 40 launches of the 64^3 workload's factor GEMM
GEMM_DRAM_PER_ALGO_BYTE = 0.386


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="lrs", choices=["lrs", "reference"])
    p.add_argument("--grid", type=int, default=64)
    p.add_argument("--leaf", type=int, default=64)
    p.add_argument("--eps", default="1e-2,1e-4,1e-6")
    p.add_argument("--nrhs", type=int, default=16)
    p.add_argument("--tol", type=float, default=1e-10)
    p.add_argument("--restart", type=int, default=30)
    p.add_argument("--maxit", type=int, default=300)
    p.add_argument("--sample-grid", type=int, default=16,
                   help="oracle sample grid side of the reference arm's steps (--impl reference)")
    p.add_argument("--cpu-grid", type=int, default=64, help="oracle grid side of the CPU baseline (default run)")
    p.add_argument("--cpu-eps", default="1e-2", help="eps values the CPU baseline's oracle runs")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--side-steps", type=int, default=5,
                   help="steps of the e2e and precision-form repeats (at most --steps)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--family", default="poisson", choices=["poisson", "varcoef"],
                   help="3D 7-point Poisson, or variable-coefficient diffusion (phi = 10^U(-3,3), seed 1)")
    p.add_argument("--gemm", default="auto", choices=["auto", "fp64", "emu"],
                   help="engine of the FP64 block products: emulated on the tensor cores (auto, emu) or FP64 FMAs")
    p.add_argument("--no-fma-form", action="store_true",
                   help="skip the one-step comparison with the FP64 products on FP64 FMAs")
    p.add_argument("--gemm-case", default="",
                   help="M,N,K: time one block product per engine (lrs_block_gemm) instead of the workload")
    p.add_argument("--gemm-engines", default="fp64,emu,tf32", help="engines --gemm-case times")
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                   help="fp32: the precision form (block products in FP32, the rest FP64)")
    p.add_argument("--no-precision-form", action="store_true",
                   help="skip the precision form's extra measurement after the FP64 form's")
    p.add_argument("--no-latency", action="store_true", help="skip the repeated-solve latency measurement")
    p.add_argument("--latency-repeats", type=int, default=20)
    p.add_argument("--no-batched-form", action="store_true", help="skip the batched-form measurement")
    p.add_argument("--no-varcoef", action="store_true",
                   help="skip the 128^3 variable-coefficient precision-form comparison")
    p.add_argument("--varcoef-grid", type=int, default=128)
    p.add_argument("--batch-count", type=int, default=256, help="instances of the batched workload")
    p.add_argument("--batch-group", type=int, default=64, help="instances factored together (one plan)")
    p.add_argument("--batch-groups", type=int, default=4,
                   help="groups timed (default 4: all 256 instances in groups of 64)")
    p.add_argument("--batch-eps", type=float, default=1e-2)
    p.add_argument("--serving", action="store_true",
                   help="run only the serving form's request stream (its own JSON line)")
    p.add_argument("--no-serving", action="store_true", help="skip the serving section of the default line")
    p.add_argument("--serving-requests", type=int, default=600)
    p.add_argument("--serving-rate", type=float, default=2.5, help="request arrivals per second (Poisson)")
    p.add_argument("--serving-sides", default="32,48,64,80,96")
    p.add_argument("--serving-eps", type=float, default=1e-2)
    p.add_argument("--serving-budget-gib", type=float, default=200.0,
                   help="factor bytes the server admits (the rest of the device holds solve workspaces)")
    p.add_argument("--serving-precision", default="tf32", choices=["fp64", "tf32"],
                   help="form of the served factorizations (tf32: the precision form, FP32 storage)")
    p.add_argument("--serving-workers", type=int, default=4)
    p.add_argument("--serving-batch-rhs", type=int, default=16)
    p.add_argument("--serving-seed", type=int, default=11)
    return p.parse_args(argv)


# ------------------------------------------------------------- replicas (N > 1)
def max_over_ranks(x, world, device):
    """The largest value of x over the ranks (the slowest replica sets the time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms):
    """Whole-job throughput: every replica's units over the slowest replica's time."""
    return world * units_per_rank / (ms / 1e3)


def make_matrix(family, g):
    import workloads as w
    return w.poisson3d(g, g, g) if family == "poisson" else w.varcoef3d(g, g, g, seed=1)


def workload(args):
    import workloads as w
    A = make_matrix(args.family, args.grid)
    B = w.rhs_uniform(A.n, range(1, args.nrhs + 1))
    return A, B


def family_name(args):
    return ("3D 7-point Poisson" if args.family == "poisson"
            else "3D 7-point variable-coefficient diffusion (phi log-uniform in [1e-3, 1e3], seed 1)")


def describe(args, n, eps_list):
    form = "FP64 form" if args.precision == "fp64" else "precision form (block products FP32, rest FP64)"
    return (f"{family_name(args)} {args.grid}^3 (n={n}, Dirichlet), leaf {args.leaf} by coordinate bisection, "
            f"eps sweep {{{', '.join(f'{e:g}' for e in eps_list)}}}, {args.nrhs} uniform[-1,1] RHS (seeds 1..{args.nrhs}), "
            f"GMRES({args.restart}) right-preconditioned to rel-res {args.tol:g}, {form}")


def precision_code(args):
    import paper_1510_07363_gb300 as lrs
    return lrs.PREC_FP64 if args.precision == "fp64" else lrs.PREC_FP32


def gemm_code(args):
    import paper_1510_07363_gb300 as lrs
    return {"auto": lrs.GEMM_AUTO, "fp64": lrs.GEMM_FP64, "emu": lrs.GEMM_EMU}[args.gemm]


# --------------------------------------------------------------------- oracle
def oracle_sample(args, eps_list, g=None):
    """The FP64 CPU oracle (single thread) on grid side g of the workload
    family (default: the reference arm's sample side)."""
    import oracle
    import workloads as w
    g = args.sample_grid if g is None else g
    A = make_matrix(args.family, g)
    B = w.rhs_uniform(A.n, range(1, args.nrhs + 1))
    t0 = time.perf_counter()
    o = oracle.Oracle(A, leaf_size=args.leaf)
    t_an = time.perf_counter() - t0
    t0 = time.perf_counter()
    iters = []
    for eps in eps_list:
        o.factor(eps)
        _, its, rel, st = o.gmres(B, restart=args.restart, maxit=args.maxit, tol=args.tol)
        iters.append(int(its.max()))
    t = time.perf_counter() - t0
    units = len(eps_list) * A.n * args.nrhs
    return {
        "value": units / t, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
        "sample": (f"{family_name(args)} {g}^3 (n={A.n}), leaf {args.leaf}, "
                   f"eps {{{', '.join(f'{e:g}' for e in eps_list)}}}, {args.nrhs} RHS, "
                   f"GMRES({args.restart}) to {args.tol:g}; single-threaded FP64 oracle, {t:.1f} s "
                   f"(analysis {t_an:.2f} s excluded), max GMRES iterations per eps {iters}"),
        "seconds": t,
    }


def cpu_baseline_job(argv):
    """Runs in a spawned process: the oracle on the CPU-baseline configuration."""
    args = parse(argv)
    import oracle
    oracle.build()
    return oracle_sample(args, [float(e) for e in args.cpu_eps.split(",")], g=args.cpu_grid)


def start_cpu_baseline(argv):
    """Starts the CPU baseline in a spawned process (before any GPU call), so
    that it overlaps the GPU measurements; returns (pool, async result)."""
    import multiprocessing as mp
    pool = mp.get_context("spawn").Pool(1)
    return pool, pool.apply_async(cpu_baseline_job, (argv,))


def run_reference(args, rank, world):
    eps_list = [float(e) for e in args.eps.split(",")]
    if rank != 0:
        return
    import oracle
    oracle.build()
    times = []
    base = None
    for step in range(args.warmup + args.steps):
        base = oracle_sample(args, eps_list)
        if step >= args.warmup:
            times.append(base["seconds"])
    t = float(np.mean(times))
    g = args.sample_grid
    units = len(eps_list) * g ** 3 * args.nrhs
    value = units / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": describe(args, args.grid ** 3, eps_list) + f"; timed on the {g}^3 sample",
                   "n": args.grid ** 3, "nrhs": args.nrhs, "eps": eps_list},
        "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                         "sample": base["sample"]},
        "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self, device_index):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != str(device_index):
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- batched form
def run_batched(args, lrs, torch, stream, dev, world):
    """The batched form: independent 2D upwind convection-diffusion matrices
    (seeded: side uniform in [64, 512], direction uniform on the circle, Peclet
    uniform in [1, 100]), factored together one group of args.batch_group
    instances at a time (one lrs_analyze_batch plan, one factorization whose
    every level covers all the group's instances) and solved by one GMRES per
    instance (one uniform[-1,1] right-hand side each), FP64 form and precision
    form.  A group of 64 needs about 80 GiB of factor storage, so the full
    256-instance set runs as four groups; by default the first group is timed."""
    import workloads as w
    ngroups = max(1, min(args.batch_groups, -(-args.batch_count // args.batch_group)))
    groups = []
    analyze_s = 0.0
    for g in range(ngroups):
        lo, hi = g * args.batch_group, min(args.batch_count, (g + 1) * args.batch_group)
        As = w.convdiff2d_batch(args.batch_count, first=lo, stop=hi)
        t0 = time.perf_counter()
        plan = lrs.lrs_analyze_batch(As, leaf_size=args.leaf)
        analyze_s += time.perf_counter() - t0
        val = torch.tensor(np.concatenate([A.val for A in As]), device=dev)
        B = torch.tensor(np.concatenate([w.rhs_uniform(A.n, [lo + k + 1])[:, 0] for k, A in enumerate(As)]),
                         device=dev)
        groups.append((plan, val, B, [A.n for A in As]))
    n_total = sum(sum(g[3]) for g in groups)
    out = {"instances": sum(len(g[3]) for g in groups), "of": args.batch_count, "group": args.batch_group,
           "unknowns": n_total, "eps": args.batch_eps, "analyze_s": analyze_s, "unit": "unknowns/s"}

    def one(group, prec, rec=None):
        plan, val, B, sizes = group
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        f = lrs.lrs_factor(plan, val, args.batch_eps, stream=stream, precision=prec, gemm=gemm_code(args))
        e1.record(stream)
        X, info, its = f.solve(B, restart=args.restart, maxit=args.maxit, tol=args.tol)
        e2.record(stream)
        e2.synchronize()
        if rec is not None:
            st = f.stats()
            rec.append({"factor_ms": e0.elapsed_time(e1), "solve_ms": e1.elapsed_time(e2),
                        "iters_min": int(its.min()), "iters_max": int(its.max()), "rel_res_max": info.rel_res,
                        "status": lrs.status_string(info.status), "factor_gib": st["factor_bytes"] / 2 ** 30,
                        "host_ms": st["host_ms"], "host_wait_ms": st["host_wait_ms"],
                        "host_elim_ms": st["host_elim_ms"], "host_merge_ms": st["host_merge_ms"],
                        "host_compress_ms": st["host_compress_ms"],
                        "max_rank": st["max_rank"], "max_pivot": st["max_pivot"]})
        del f, X

    for name, prec in (("fp64", lrs.PREC_FP64), ("precision_form", lrs.PREC_FP32)):
        one(groups[0], prec)                             # warm-up
        torch.cuda.synchronize()
        recs = []
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for g in groups:
            one(g, prec, recs)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
        out[name] = {"value": job_value(n_total, world, ms), "ms": ms, "groups": recs}
    out["vs_fp64_form"] = out["precision_form"]["value"] / out["fp64"]["value"]
    return out


# ------------------------------------------- variable-coefficient precision form
def run_varcoef(args, lrs, torch, stream, dev, world):
    """3D variable-coefficient diffusion (phi log-uniform in [1e-3, 1e3], seed
    1, Dirichlet) on a --varcoef-grid^3 grid, leaf 64, eps = 1e-2, one
    uniform[-1,1] right-hand side, GMRES(30) to 1e-10: the FP64 form and the
    precision form, each one warm-up run then one timed factor + solve."""
    import workloads as w
    g = args.varcoef_grid
    A = w.varcoef3d(g, g, g, seed=1)
    t0 = time.perf_counter()
    plan = lrs.lrs_analyze(A, leaf_size=args.leaf)
    analyze_s = time.perf_counter() - t0
    val = torch.tensor(A.val, device=dev)
    b = torch.tensor(w.rhs_uniform(A.n, [1])[:, 0], device=dev)
    out = {"workload": f"3D 7-point variable-coefficient diffusion {g}^3 (n={A.n}, phi log-uniform in "
                       f"[1e-3, 1e3], seed 1, Dirichlet), leaf {args.leaf}, eps 1e-2, 1 uniform[-1,1] RHS, "
                       f"GMRES({args.restart}) to {args.tol:g}",
           "n": A.n, "analyze_s": analyze_s, "unit": "unknowns/s"}
    for name, prec in (("fp64", lrs.PREC_FP64), ("precision_form", lrs.PREC_FP32)):
        rec = None
        for rep in range(2):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            f = lrs.lrs_factor(plan, val, 1e-2, stream=stream, precision=prec, gemm=gemm_code(args))
            e1.record(stream)
            x, info, its = f.solve(b, restart=args.restart, maxit=args.maxit, tol=args.tol)
            e2.record(stream)
            e2.synchronize()
            ms = max_over_ranks(e0.elapsed_time(e2), world, dev)
            st = f.stats()
            rec = {"value": job_value(A.n, world, ms), "ms": ms, "factor_ms": e0.elapsed_time(e1),
                   "solve_ms": e1.elapsed_time(e2), "iters": int(its.max()), "rel_res": info.rel_res,
                   "status": lrs.status_string(info.status), "max_rank": st["max_rank"],
                   "factor_gib": st["factor_bytes"] / 2 ** 30}
            del f, x
        out[name] = rec
    out["vs_fp64_form"] = out["precision_form"]["value"] / out["fp64"]["value"]
    return out


# ------------------------------------------------------------- serving form
def serving_requests(count, rate, nsides, seed):
    """Seeded request stream: Poisson arrivals at `rate` per second; 90% are
    solves of 1-8 uniform[-1,1] right-hand sides against one of the 8 resident
    factors, 10% new factorizations (a side index and a family: 0 Poisson,
    1 variable-coefficient diffusion).  Entries (kind, arrival s, a, b)."""
    import workloads as w
    u = w.uniform01(seed, 4 * count)
    t, out = 0.0, []
    for i in range(count):
        t += -np.log1p(-u[4 * i]) / rate
        if u[4 * i + 1] < 0.9:
            out.append(("solve", t, int(8 * u[4 * i + 2]), 1 + int(8 * u[4 * i + 3])))
        else:
            out.append(("factor", t, int(nsides * u[4 * i + 2]), int(2 * u[4 * i + 3])))
    return out


def run_serving(args, executor=None):
    """The serving form under a request stream: 8 factorizations of 3D Poisson /
    variable-coefficient diffusion operators (sides from --serving-sides) made
    resident first, then --serving-requests requests dispatched at their
    arrival times from one thread while another collects them in order (a new
    factorization is evicted once built, as a tenant that leaves).  Latencies
    are the server's (queue + run) per request; throughput counts the solves
    over the stream's wall time."""
    import queue
    import threading

    import workloads as w
    import paper_1510_07363_gb300 as lrs
    sides = [int(x) for x in args.serving_sides.split(",")]
    sprec = lrs.PREC_FP64 if args.serving_precision == "fp64" else lrs.PREC_TF32
    shapes = {}

    def shape(si, fam):
        if (si, fam) not in shapes:
            g = sides[si]
            A = w.poisson3d(g, g, g) if fam == 0 else w.varcoef3d(g, g, g, seed=1)
            shapes[(si, fam)] = (A, lrs.lrs_analyze(A, leaf_size=args.leaf))
        return shapes[(si, fam)]

    u = w.uniform01(args.serving_seed + 1, 16)
    initial = [(int(len(sides) * u[2 * k]), int(2 * u[2 * k + 1])) for k in range(8)]
    budget = int(args.serving_budget_gib * 2 ** 30)
    # a guard on the residents' size: an FP64 factor at eps = 1e-2 holds up to
    # ~64 KB per unknown on these operators, the precision form's FP32 one half that
    per_unknown0 = 65536 if sprec == lrs.PREC_FP64 else 32768
    if sum(per_unknown0 * sides[si] ** 3 for si, _ in initial) > budget:
        raise RuntimeError(f"the 8 resident factorizations ({per_unknown0} bytes per unknown) exceed "
                           "--serving-budget-gib")
    srv = lrs.Server(budget, workers=args.serving_workers, max_batch_rhs=args.serving_batch_rhs,
                     executor=executor)
    try:
        resident = []
        for sh in initial:
            A, plan = shape(*sh)
            resident.append((srv.factor(plan, A.val, args.serving_eps, precision=sprec), A))
        factor_bytes = []
        for t, _ in resident:
            _, info = srv.wait(t)
            if info.status != 0:
                raise RuntimeError(f"resident factorization failed: {lrs.status_string(info.status)}")
            factor_bytes.append(info.bytes)
        # new tenants reserve the residents' largest bytes per unknown; one that
        # cannot fit beside the residents even alone is refused, not queued
        per_unknown = max(b / A.n for b, (_, A) in zip(factor_bytes, resident)) * 1.25 + 1.0
        room = budget - sum(factor_bytes)
        reqs = serving_requests(args.serving_requests, args.serving_rate, len(sides), args.serving_seed)
        for kind, _, a, b in reqs:
            if kind == "factor":
                shape(a, b)                                 # analysis is not part of the stream
        rhs = {}
        inbox = queue.Queue()
        results = {"solve": [], "factor": [], "failed": 0, "batched": 0, "unknowns": 0, "refused": 0,
                   "fail_status": {}}

        def collect():
            while True:
                item = inbox.get()
                if item is None:
                    return
                kind, t, nrhs, n = item
                _, info = srv.wait(t)
                if info.status != 0:
                    results["failed"] += 1
                    key = f"{kind}: {lrs.status_string(info.status)}"
                    results["fail_status"][key] = results["fail_status"].get(key, 0) + 1
                    continue
                results[kind].append(info.queue_ms + info.run_ms)
                if kind == "factor":
                    srv.evict(t)
                else:
                    results["batched"] += info.batch_rhs > nrhs
                    results["unknowns"] += n * nrhs

        th = threading.Thread(target=collect)
        th.start()
        t0 = time.perf_counter()
        for kind, at, a, b in reqs:
            delay = at - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            if kind == "solve":
                ft, A = resident[a]
                if (a, b) not in rhs:
                    rhs[(a, b)] = w.rhs_uniform(A.n, range(1, b + 1))
                inbox.put(("solve", srv.solve(ft, rhs[(a, b)], tol=args.tol, restart=args.restart,
                                              maxit=args.maxit), b, A.n))
            else:
                A, plan = shape(a, b)
                reserve = int(per_unknown * A.n)
                if reserve > room:
                    results["refused"] += 1
                    continue
                inbox.put(("factor", srv.factor(plan, A.val, args.serving_eps, precision=sprec, reserve_bytes=reserve),
                           0, A.n))
        inbox.put(None)
        th.join()
        wall = time.perf_counter() - t0
    finally:
        srv.close()
    sol, fac = np.array(results["solve"]), np.array(results["factor"])
    pct = lambda v, q: float(np.percentile(v, q)) if v.size else None
    return {
        "requests": len(reqs), "solves": int(sol.size), "factorizations": int(fac.size),
        "failed": results["failed"], "failed_by_status": results["fail_status"],
        "refused_no_room": results["refused"], "wall_s": wall,
        "solves_per_s": sol.size / wall,
        "unknowns_per_s": results["unknowns"] / wall,
        "solve_ms_p50": pct(sol, 50), "solve_ms_p99": pct(sol, 99),
        "factor_ms_p50": pct(fac, 50), "factor_ms_p99": pct(fac, 99),
        "merged_solves": results["batched"], "resident_gib": sum(factor_bytes) / 2 ** 30,
        "sides": sides, "eps": args.serving_eps, "rate_per_s": args.serving_rate,
        "precision": args.serving_precision, "budget_gib": args.serving_budget_gib, "workers": args.serving_workers,
    }


# --------------------------------------------------------------------- GPU arm
def run_lrs(args, rank, world, local_rank, cpu_job=None):
    import torch
    import torch.distributed as dist

    import paper_1510_07363_gb300 as lrs
    from paper_1510_07363_gb300 import build as lrs_build

    torch.cuda.set_device(local_rank)
    if rank == 0:
        lrs_build.build()
    if world > 1:
        dist.barrier()
    lrs.load()
    eps_list = [float(e) for e in args.eps.split(",")]
    A, B = workload(args)
    t0 = time.perf_counter()
    plan = lrs.lrs_analyze(A, leaf_size=args.leaf)
    analyze_s = time.perf_counter() - t0
    dev = torch.device("cuda", local_rank)
    val_d = torch.tensor(A.val, device=dev)
    B_d = torch.tensor(B, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def step(record=None, profile=False, precision=None, gemm=None):
        prof = {}
        prec = precision_code(args) if precision is None else precision
        gm = gemm_code(args) if gemm is None else gemm
        for eps in eps_list:
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            f = lrs.lrs_factor(plan, val_d, eps, stream=stream, profile=profile, precision=prec, gemm=gm)
            e1.record(stream)
            X, info, its = f.solve(B_d, restart=args.restart, maxit=args.maxit, tol=args.tol)
            e2.record(stream)
            e2.synchronize()
            if record is not None:
                st = f.stats()
                record.append({"eps": eps, "factor_ms": e0.elapsed_time(e1), "gmres_ms": e1.elapsed_time(e2),
                               "iters_max": int(its.max()), "iters_min": int(its.min()),
                               "rel_res_max": info.rel_res, "status": lrs.status_string(info.status),
                               "max_rank": st["max_rank"], "max_pivot": st["max_pivot"], "ext_n": st["ext_n"],
                               "factor_gflop": st["flops_factor"] / 1e9, "spectrum_gflop": st["eig_flops"] / 1e9,
                               "factor_gib": st["factor_bytes"] / 2 ** 30, "batches": st["n_batches"],
                               "spectrum_phase_gcycles": [c / 1e9 for c in st["eig_cycles"]],
                               "spectrum_phase_lead_ms": list(st["eig_lead_ms"]),
                               "host_ms": st["host_ms"], "host_wait_ms": st["host_wait_ms"],
                               "host_elim_ms": st["host_elim_ms"],
                               "depth": st["depth"]})
            if profile:
                for k, v in lrs.lrs_factor_profile(f).items():
                    acc = prof.setdefault(k, {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0})
                    for kk in acc:
                        acc[kk] += v[kk]
            del f, X
        flush.zero_()
        return prof

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    records, profs = [], []
    clock_path = os.path.join(tempfile.gettempdir(), f"lrs_bench_clocks_rank{rank}_{os.getpid()}.csv")
    with ClockSampler(clock_path) as clocks:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(args.steps):
            profs.append(step(records, profile=True))
        end.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = max_over_ranks(start.elapsed_time(end) / args.steps, world, dev)
    units = len(eps_list) * A.n * args.nrhs
    value = job_value(units, world, ms)

    # repeated-solve and apply latencies on the first eps's factor, for the
    # FP64 form and the precision form (CUDA events), and the apply's roofline:
    # bytes of stored blocks read per application over its p50 time
    latency = None
    if not args.no_latency:
        eps0 = eps_list[0]
        hbm = measured_peak("hbm_gbs", 6800.0)
        latency = {"eps": eps0, "repeats": args.latency_repeats, "nrhs": args.nrhs}
        for name, prec in (("fp64", lrs.PREC_FP64), ("precision_form", lrs.PREC_FP32)):
            f = lrs.lrs_factor(plan, val_d, eps0, stream=stream, precision=prec, gemm=gemm_code(args))
            solve_ms, apply_ms, apply1_ms = [], [], []
            b1 = B_d[:, :1].contiguous()
            for reps, out, arg, fn in ((args.latency_repeats, solve_ms, B_d, "solve"),
                                       (args.latency_repeats, apply_ms, B_d, "apply"),
                                       (args.latency_repeats, apply1_ms, b1, "apply")):
                for _ in range(reps):
                    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a0.record(stream)
                    if fn == "solve":
                        f.solve(arg, restart=args.restart, maxit=args.maxit, tol=args.tol)
                    else:
                        f.apply(arg)
                    a1.record(stream)
                    a1.synchronize()
                    out.append(a0.elapsed_time(a1))
            ab = f.stats()["apply_bytes"]
            p50 = float(np.percentile(apply_ms, 50))
            p50_1 = float(np.percentile(apply1_ms, 50))
            latency[name] = {
                "solve_ms_p50": float(np.percentile(solve_ms, 50)), "solve_ms_p99": float(np.percentile(solve_ms, 99)),
                "apply_ms_p50": p50, "apply_ms_p99": float(np.percentile(apply_ms, 99)),
                "apply1_ms_p50": p50_1,
                "apply_roofline": {"bound": "hbm", "bytes_per_apply": ab,
                                   "achieved_gbs": ab / (p50 / 1e3) / 1e9, "achieved_gbs_1rhs": ab / (p50_1 / 1e3) / 1e9,
                                   "peak": hbm[0], "peak_source": hbm[1], "unit": "GB/s",
                                   "frac": ab / (p50 / 1e3) / 1e9 / hbm[0],
                                   "frac_1rhs": ab / (p50_1 / 1e3) / 1e9 / hbm[0]}}
            del f
        latency["solve_ms_p50"] = latency["fp64"]["solve_ms_p50"]
        latency["solve_ms_p99"] = latency["fp64"]["solve_ms_p99"]

    side_steps = max(1, min(args.steps, args.side_steps))
    # the precision form (block products on the tensor cores) on the same
    # workload, after the FP64 form's timed region: one warm-up step, then
    # side_steps timed, with the same per-launch profiling as the FP64 form
    precision_form = None
    if args.precision == "fp64" and not args.no_precision_form:
        step(precision=lrs.PREC_FP32)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        precs, pprofs = [], []
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(side_steps):
            pprofs.append(step(precs, profile=True, precision=lrs.PREC_FP32))
        p1.record(stream)
        torch.cuda.synchronize()
        pms = max_over_ranks(p0.elapsed_time(p1) / side_steps, world, dev)
        ptotal = {}
        for p in pprofs:
            for k, v in p.items():
                acc = ptotal.setdefault(k, {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0})
                for kk in acc:
                    acc[kk] += v[kk]
        tc = ptotal.get("factor_gemm_f32", {"ms": 0.0, "flops": 0.0, "launches": 0})
        precision_form = {
            "value": job_value(units, world, pms), "unit": "unknowns/s", "ms_per_step": pms, "steps": side_steps,
            "vs_fp64_form": ms / pms,
            "what": "Schur updates, A_pp^-1 A_pk, projections and (eps >= 1e-2) Gram matrices on the tensor cores "
                    "(tcgen05 kind::tf32, TF32 head + tail split, FP32 accumulation in tensor memory); inverses, "
                    "spectra, rank decisions, traversals and GMRES FP64",
            "tensor_gemm": {"launches": tc["launches"], "ms_per_step": tc["ms"] / side_steps,
                            "tflops_fp32_equivalent": tc["flops"] / max(tc["ms"], 1e-9) / 1e9,
                            "tflops_tf32_issued": 3 * tc["flops"] / max(tc["ms"], 1e-9) / 1e9},
            "kernel_classes": {k: {"launches": v["launches"], "ms_per_step": v["ms"] / side_steps,
                                   "gflop_per_step": v["flops"] / 1e9 / side_steps}
                               for k, v in ptotal.items()},
            "per_eps": [{"eps": r["eps"], "factor_ms": r["factor_ms"], "solve_ms": r["gmres_ms"],
                         "iters_max": r["iters_max"], "rel_res_max": r["rel_res_max"], "status": r["status"]}
                        for r in precs]}

    # the same workload with the FP64 block products on FP64 FMAs (the engine
    # the emulation replaces): one step, unprofiled, for the comparison
    fma_form = None
    if args.precision == "fp64" and not args.no_fma_form and args.gemm != "fp64":
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        step(gemm=lrs.GEMM_FP64)
        q1.record(stream)
        torch.cuda.synchronize()
        qms = max_over_ranks(q0.elapsed_time(q1), world, dev)
        fma_form = {"value": job_value(units, world, qms), "unit": "unknowns/s", "ms_per_step": qms, "steps": 1,
                    "what": "FP64 form with the block products on FP64 FMAs (CUDA cores) instead of emulated "
                            "on the tensor cores",
                    "emulated_speedup": qms / ms}

    # the batched form runs after every headline measurement; a failure there
    # (say, too little device memory for a group) is reported in its entry
    # rather than costing the line
    batched_form = None
    if not args.no_batched_form:
        try:
            batched_form = run_batched(args, lrs, torch, stream, dev, world)
        except Exception as exc:                      # noqa: BLE001 -- reported, not hidden
            batched_form = {"error": f"{type(exc).__name__}: {exc}"}

    varcoef = None
    if not args.no_varcoef:
        try:
            varcoef = run_varcoef(args, lrs, torch, stream, dev, world)
        except Exception as exc:                      # noqa: BLE001 -- reported, not hidden
            varcoef = {"error": f"{type(exc).__name__}: {exc}"}

    # per-kernel-class profile over the timed region
    total = {}
    for p in profs:
        for k, v in p.items():
            acc = total.setdefault(k, {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0})
            for kk in acc:
                acc[kk] += v[kk]
    launches = int(sum(v["launches"] for v in total.values()))
    # (the spectrum class's flops: the device counter of the spectra, lrs_stats.eig_flops,
    # plus the super-node inverses that run in the same launches)
    ktime = sum(v["ms"] for v in total.values())

    def class_roofline(name):
        d = total[name]
        if name in ("apply_gemm", "spmv", "vector", "copy", "assemble") and d["flops"] / max(d["bytes"], 1) < 0.5:
            ach = d["bytes"] / (d["ms"] / 1e3) / 1e9
            peak = measured_peak("hbm_gbs", 6800.0)
            r = {"bound": "hbm", "kernel_class": name, "achieved": ach, "peak": peak[0], "unit": "GB/s",
                 "frac": ach / peak[0], "peak_source": peak[1]}
        elif name == "factor_gemm_emu":
            # FP64 products emulated on the tensor cores: 36 BF16 digit products per
            # FP64 multiply-add, so the BF16 work is 36x the FP64 algorithmic flops
            # (a lower bound: tile padding adds more); against the sustained BF16 peak
            ach = d["flops"] / (d["ms"] / 1e3) / 1e9
            peak = measured_peak("bf16_tflops_sustained", 1700.0)
            r = {"bound": "tensor", "kernel_class": name, "achieved": 36 * ach / 1e3, "peak": peak[0],
                 "unit": "TFLOP/s", "frac": 36 * ach / 1e3 / peak[0], "peak_source": peak[1] + ", bf16 sustained",
                 "fp64_equivalent_tflops": ach / 1e3, "vs_fp64_pipe": ach / FP64_PEAK_GFLOPS}
        elif name == "factor_gemm_f32":
            ach = d["flops"] / (d["ms"] / 1e3) / 1e9
            r = {"bound": "alu", "kernel_class": name, "achieved": ach / 1e3, "peak": FP32_PEAK_GFLOPS / 1e3,
                 "unit": "TFLOP/s", "frac": ach / FP32_PEAK_GFLOPS,
                 "peak_source": "FP32 FMA pipe, derived: 152 SMs x 128 FMA/clk x 2 flop x 2.06 GHz"}
        else:
            ach = d["flops"] / (d["ms"] / 1e3) / 1e9
            r = {"bound": "alu", "kernel_class": name, "achieved": ach / 1e3, "peak": FP64_PEAK_GFLOPS / 1e3,
                 "unit": "TFLOP/s", "frac": ach / FP64_PEAK_GFLOPS,
                 "peak_source": "FP64 FMA pipe, derived: 152 SMs x 2 FMA/clk x 2 flop x 2.06 GHz "
                                "(measured 1.19 TFLOP/s at 1.96 GHz)"}
        r["traffic"] = None
        if name == "factor_gemm":
            r["traffic"] = GEMM_DRAM_PER_ALGO_BYTE * d["bytes"] / max(d["launches"], 1)
            r["traffic_unit"] = "bytes per launch"
            r["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of 40 full-size "
                                   "launches: 0.386 of their algorithmic bytes, scaled to this "
                                   "region's mean algorithmic bytes per launch")
        r["launches"] = d["launches"]
        r["avg_launch_ms"] = d["ms"] / max(d["launches"], 1)
        r["share_of_kernel_time"] = d["ms"] / ktime
        return r

    dom = max(total, key=lambda k: total[k]["ms"]) if total else None
    roofline = class_roofline(dom) if dom else None
    # every class above 5% of the kernel time, for the whole picture
    roofline_by_class = {k: class_roofline(k) for k in total if ktime > 0 and total[k]["ms"] > 0.05 * ktime}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        val_h = torch.tensor(A.val).pin_memory()
        B_h = torch.tensor(np.ascontiguousarray(B.T)).pin_memory()      # nrhs x n row-major = n x nrhs col-major
        X_h = torch.empty_like(B_h).pin_memory()
        vh, bh, xh = val_h.numpy(), B_h.numpy(), X_h.numpy()
        import ctypes
        lib = lrs.load()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(side_steps):
            for eps in eps_list:
                f = lrs.lrs_factor(plan, vh, eps, stream=stream, precision=precision_code(args),
                                   gemm=gemm_code(args))
                opts = lrs._SolveOpts(args.restart, args.maxit, args.tol)
                info = lrs.SolveInfo()
                lib.lrs_solve(f._h, ctypes.c_void_p(bh.ctypes.data), ctypes.c_void_p(xh.ctypes.data), args.nrhs, 0,
                              ctypes.byref(opts), ctypes.byref(info))
                del f
        torch.cuda.synchronize()
        te = max_over_ranks((time.perf_counter() - t0) / side_steps, world, dev)
        e2e = {"value": world * units / te, "unit": "unknowns/s",
               "h2d_bytes_per_step": len(eps_list) * (A.nnz * 8 + A.n * args.nrhs * 8),
               "d2h_bytes_per_step": len(eps_list) * A.n * args.nrhs * 8,
               "ms_per_step": te * 1e3, "steps": side_steps}

    # the serving form (each rank serves its own stream), after everything else;
    # its executor allocates outside PyTorch's caching allocator, so the cache
    # the earlier sections filled is returned to the device first
    serving = None
    if not args.no_serving:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        try:
            serving = run_serving(args)
        except Exception as exc:                      # noqa: BLE001 -- reported, not hidden
            serving = {"error": f"{type(exc).__name__}: {exc}"}

    clk = clocks.summary(local_rank)
    if rank != 0:
        return
    cpu = None
    if cpu_job is not None:
        pool, res = cpu_job
        try:
            cb = res.get(timeout=3600)
            cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
            cpu["overlapped"] = "ran in a spawned process on one host core during the GPU measurements"
        except Exception as exc:                      # noqa: BLE001 -- reported, not hidden
            cpu = {"error": f"{type(exc).__name__}: {exc}"}
        finally:
            pool.terminate()
    per_eps = {}
    for r in records:
        d = per_eps.setdefault(r["eps"], [])
        d.append(r)
    summary = []
    for eps, rs in per_eps.items():
        gm = np.array([r["gmres_ms"] for r in rs])
        fm = np.array([r["factor_ms"] for r in rs])
        last = rs[-1]
        summary.append({**{k: last[k] for k in last if k not in ("factor_ms", "gmres_ms")},
                        "factor_ms_p50": float(np.median(fm)), "solve_ms_p50": float(np.percentile(gm, 50)),
                        "solve_ms_p99": float(np.percentile(gm, 99))})
    line = {
        "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": describe(args, A.n, eps_list), "n": A.n, "nnz": A.nnz, "nrhs": args.nrhs,
                   "eps": eps_list, "leaf": args.leaf, "depth": plan_depth(records),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "256 MiB buffer written between steps (inside the timed region); factor working set > L2",
                   "analyze_s": analyze_s, "per_eps": summary,
                   "kernel_classes": {k: {"launches": v["launches"], "ms": v["ms"],
                                          "gflop": v["flops"] / 1e9, "gbyte": v["bytes"] / 1e9}
                                      for k, v in total.items()}},
        "roofline": roofline, "roofline_by_class": roofline_by_class, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
        "precision_form": precision_form, "batched_form": batched_form, "latency": latency,
        "serving": serving, "varcoef_precision": varcoef, "fp64_fma_form": fma_form,
        "gemm_engine": args.gemm,
    }
    print(json.dumps(line), flush=True)


def run_gemm_case(args):
    """One block product C = op(A) op(B) of the given size per engine, through
    lrs_block_gemm on seeded normal data (operands larger than L2 at the
    profiling size 4096^3): median kernel time of `steps` calls after `warmup`."""
    import torch
    import paper_1510_07363_gb300 as lrs
    lrs.load()
    M, N, K = (int(x) for x in args.gemm_case.split(","))
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.randn(K, M, device="cuda", dtype=torch.float64, generator=g).t()     # M x K, column-major
    B = torch.randn(N, K, device="cuda", dtype=torch.float64, generator=g).t()     # K x N, column-major
    C = torch.zeros(N, M, device="cuda", dtype=torch.float64).t()
    out = {"gemm_case": [M, N, K], "unit": "TFLOP/s (FP64-equivalent, 2 M N K per product)"}
    for name in [e for e in args.gemm_engines.split(",") if e]:
        eng = {"fp64": lrs.GEMM_FP64, "emu": lrs.GEMM_EMU, "tf32": lrs.GEMM_TF32}[name]
        for _ in range(args.warmup):
            lrs.lrs_block_gemm(eng, A, B, C)
        ts = sorted(lrs.lrs_block_gemm(eng, A, B, C) for _ in range(max(1, args.steps)))
        ms = ts[len(ts) // 2]
        out[name] = {"ms": ms, "tflops": 2.0 * M * N * K / (ms / 1e3) / 1e12}
    print(json.dumps(out), flush=True)


def plan_depth(records):
    return records[0]["depth"] if records else None


def measured_peak(key, fallback):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = json.load(f).get(key)
        if v:
            return float(v), "measured (MEASURED_PEAKS.json)"
    except (OSError, ValueError):
        pass
    return fallback, "fallback"


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    cpu_job = None
    if args.gemm_case:
        if rank == 0:
            run_gemm_case(args)
        return
    if args.impl == "lrs" and not args.serving and rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_job = start_cpu_baseline(sys.argv[1:])
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "lrs" else "gloo"
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        elif args.serving:
            if rank == 0:
                out = run_serving(args)
                print(json.dumps({"metric": "serving: p50/p99 solve latency and solves/s", "n_gpus": world,
                                  "data": "synthetic", "dtype": "f64", "serving": out}), flush=True)
        else:
            run_lrs(args, rank, world, local_rank, cpu_job)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
