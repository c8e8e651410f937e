#!/usr/bin/env python
"""Throughput of the Lloyd-preconditioned LBFGS SCVT solver on GB300.

A step is one LBFGS iteration of the whole hot path: the two-loop direction,
the line search (each trial re-bins the generators, rebuilds every Voronoi
cell and integrates it) and the accepted-pair update.  The default workload
is the 2,621,442-generator tanh-cap problem (gamma = (1/8)^4, alpha = 0.10,
beta = pi/9, x_c at 45N 270E, LBFGS memory 7, FP64) from seeded uniform
points; the metric is generator-updates/s = N x accepted iterations / s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one process per GPU) every rank solves its own
independent instance (replicas, weak scaling, no collective on the data
path); rank 0 prints one JSON line.  ``--impl reference`` times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1709_06924_gb300 import inputs as I  # noqa: E402

def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="tanh-2621442", choices=sorted(I.WORKLOADS))
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--cpu-sample-n", type=int, default=163842,
                   help="generators of the bounded oracle sample (same density)")
    p.add_argument("--cpu-sample-iters", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-other-form", action="store_true", help="skip timing the other precision form")
    p.add_argument("--no-time-to-tol", action="store_true", help="skip the time-to-tolerance runs")
    p.add_argument("--no-batched", action="store_true", help="skip the 64-problem batch")
    p.add_argument("--no-tune", action="store_true", help="keep the default tuning (no autotuner run)")
    p.add_argument("--tuning", default="",
                   help="fixed tuning instead of the autotuner, e.g. chunks=4,bin_load=8 (other fields default)")
    p.add_argument("--no-serving", action="store_true", help="skip the request-stream measurement")
    p.add_argument("--no-table1", action="store_true", help="skip the 2,562-generator method comparison")
    p.add_argument("--no-chain", action="store_true", help="skip the 2,562 -> 655,362 bisection chain")
    p.add_argument("--serve-jobs", type=int, default=32, help="jobs in the request stream")
    p.add_argument("--serve-n-hi", type=int, default=655362, help="largest job size of the request stream")
    p.add_argument("--serve-max-iter", type=int, default=100, help="iteration cap per served job")
    p.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                   help="fp64: everything in FP64; mixed: FP32 corners/quadrature, FP64 sums and LBFGS")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 10:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self):
        rows = [r for r in self.rows if self.uuid is None or self.uuid in r[1]] or self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        mx = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[4]) or 0.0) for r in rows)}


# ----------------------------------------------------------------- CPU oracle
def oracle_sample(w: I.Workload, n_sample: int, iters: int, seed: int):
    """Time the FP64 oracle's own solver on a bounded sample: the same density
    and solver settings on n_sample seeded generators, `iters` iterations."""
    import oracle
    oracle.build()
    z = I.uniform_sphere(n_sample, seed)
    t0 = time.perf_counter()
    _, rep, _ = oracle.lbfgs_solve(z, w.density, lbfgs_m=w.lbfgs_m, max_iter=iters, grad_tol=0.0)
    t = time.perf_counter() - t0
    return {"value": n_sample * rep["iters"] / t, "unit": "generator-updates/s", "cores": oracle.max_threads(),
            "kind": "oracle", "seconds": t, "iters": rep["iters"], "fevals": rep["fevals"],
            "sample": "%d seeded generators, same density and LBFGS memory, %d oracle iterations "
                      "(including the initial evaluation)" % (n_sample, rep["iters"])}


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    n = args.cpu_sample_n
    z = I.uniform_sphere(n, args.seed)
    if args.warmup > 0:
        z, _, _ = oracle.lbfgs_solve(z, w.density, lbfgs_m=w.lbfgs_m, max_iter=args.warmup, grad_tol=0.0)
    t0 = time.perf_counter()
    _, rep, _ = oracle.lbfgs_solve(z, w.density, lbfgs_m=w.lbfgs_m, max_iter=args.steps, grad_tol=0.0)
    t = time.perf_counter() - t0
    value = n * rep["iters"] / t
    cores = oracle.max_threads()
    sample = ("%d seeded generators of the %s workload's density and solver settings; %d timed oracle "
              "iterations after %d warm-up iterations (history restarts at the timed call)"
              % (n, w.name, rep["iters"], args.warmup))
    line = {
        "impl": "reference", "metric": "generator-updates/s", "value": value, "unit": "generator-updates/s",
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / max(rep["iters"], 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_generators": w.n, "sample_generators": n, "lbfgs_m": w.lbfgs_m,
                   "density": "tanh cap", "seed": args.seed},
        "cpu_baseline": {"value": value, "unit": "generator-updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "generator-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- our arm
def combine_ranks(units: float, seconds: float, device=None):
    """Whole-job numbers over replicas: units summed, time = max over ranks
    (torch.distributed; identity on a single process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(seconds)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def timed_steps(eng, z, steps):
    """K LBFGS iterations continuing the engine's state, timed with CUDA
    events on the engine's stream; returns (report, seconds)."""
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(eng.stream)
    rep = eng.lbfgs_solve(z, max_iter=steps, grad_tol=0.0, warm_start=True)
    ev1.record(eng.stream)
    torch.cuda.synchronize()
    return rep, ev0.elapsed_time(ev1) / 1e3


def parse_tuning(text):
    """'k=v,k=v' -> {k: int(v)} (empty text: {})."""
    out = {}
    for item in filter(None, (t.strip() for t in text.split(","))):
        k, v = item.split("=")
        out[k.strip()] = int(v)
    return out


def pick_tuning(args, eng, z):
    """The autotuner's choice, the default tuning (--no-tune), or the fixed
    fields of --tuning on top of the default."""
    fixed = parse_tuning(args.tuning)
    if fixed:
        eng.set_tuning(**fixed)
        return eng.tuning()
    return eng.tune(z) if not args.no_tune else eng.tuning()


def time_to_tolerance(w, z_host, local, prec, tuning, tol=1e-6, max_iter=50):
    """Wall time from the seeded start until ||grad E||_2 <= tol (the
    workload's stated criterion), with the iterate on the device (the
    tuning found once for the workload is applied, not re-searched)."""
    import torch
    from paper_1709_06924_gb300.engine import Engine
    eng = Engine(w.n, w.density, lbfgs_m=w.lbfgs_m, device=local, precision=prec)
    eng.set_tuning(**tuning)
    z = torch.from_numpy(z_host).cuda(local)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = eng.lbfgs_solve(z, max_iter=max_iter, grad_tol=tol)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    eng.close()
    return {"grad_tol": tol, "seconds": t, "iters": rep["iters"], "fevals": rep["fevals"],
            "converged": bool(rep["converged"]), "grad_norm": rep["grad_norm"],
            "grad_norm_over_F": rep["grad_norm"] / rep["energy"]}


def run_batched(args, local, prec, count=64):
    """64 independent problems (N log-uniform in [10,242, 655,362], each its own
    tanh cap) as one batch: autotuned, W warm-up and K timed lockstep LBFGS
    iterations.  Units = sum over problems of N_b x iterations."""
    import torch
    from paper_1709_06924_gb300.engine import Batch
    inst = I.sample_batched_instances(count, args.seed)
    ns = [n for n, _, _ in inst]
    zs = [I.uniform_sphere(n, sd) for n, _, sd in inst]
    bt = Batch(ns, [d for _, d, _ in inst], lbfgs_m=7, precision=prec, device=local)
    try:
        z = torch.from_numpy(np.concatenate(zs)).cuda(local)
        t0 = time.perf_counter()
        tuning = bt.tune(z)
        t_tune = time.perf_counter() - t0
        bt.lbfgs_solve(z, max_iter=args.warmup, grad_tol=0.0)
        bt.reset_stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = bt.lbfgs_solve(z, max_iter=args.steps, grad_tol=0.0, warm_start=1)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        st = bt.stats()
    finally:
        bt.close()
    units = sum(n * r["iters"] for n, r in zip(ns, reps))
    return {"problems": count, "n_total": int(sum(ns)), "n_min": int(min(ns)), "n_max": int(max(ns)),
            "precision": "mixed" if prec else "fp64", "value": units / t, "unit": "generator-updates/s",
            "seconds": t, "iters": [r["iters"] for r in reps][:4] + ["..."],
            "evaluations": st["evaluations"], "gpu_launches": st["kernel_launches"], "tuning": tuning,
            "tune_seconds": t_tune, "timing": "host wall clock around the synchronous batch solve",
            "statuses": sorted({r["status"] for r in reps})}


def serve_stream(srv, jobs, arrivals, max_iter, tol):
    """Submit job k at arrivals[k] seconds (server clock, from the first
    submission), stepping the server in between; returns per-job records."""
    t0 = srv.clock()
    ids = {}
    k = 0
    while True:
        now = srv.clock() - t0
        while k < len(jobs) and arrivals[k] <= now:
            z, dens = jobs[k]
            ids[k] = srv.submit(z, dens, max_iter=max_iter, grad_tol=tol)
            k += 1
        running, queued = srv.step()
        if running == 0 and queued == 0:
            if k == len(jobs):
                break
            time.sleep(max(0.0, min(arrivals[k] - (srv.clock() - t0), 0.05)))
    recs = []
    for j in range(len(jobs)):
        info = srv.job(ids[j])
        recs.append(info)
        srv.fetch(ids[j])
    return recs


def run_serving(args, local, prec, count=None):
    """A Poisson stream of solve requests through the continuous-batching
    server: N log-uniform in [40,962, n_hi], random tanh caps (the batched
    workloads' sampler), each job to ||grad E||_2 <= 1e-6 (at most max_iter
    iterations).  A closed-loop pass (all jobs at t = 0) measures the service
    capacity; the timed pass offers Poisson arrivals at 80 % of it."""
    from paper_1709_06924_gb300.engine import Server
    count = count or args.serve_jobs
    inst = I.sample_batched_instances(count, args.seed + 7, n_lo=40962, n_hi=args.serve_n_hi)
    jobs = [(I.uniform_sphere(n, sd), d) for n, d, sd in inst]
    max_iter, tol = args.serve_max_iter, 1e-6
    cap_n = max(4 * max(n for n, _, _ in inst), 2_000_000)
    with Server(max_generators=cap_n, max_jobs=32, precision=prec, device=local) as srv:
        closed = serve_stream(srv, jobs, [0.0] * count, max_iter, tol)
        t_closed = max(r["t_done"] for r in closed) - min(r["t_submit"] for r in closed)
        rate = 0.8 * count / t_closed
        rng = np.random.default_rng(args.seed + 11)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=count))
        arrivals -= arrivals[0]
        ev0 = srv.stats()["evaluations"]
        recs = serve_stream(srv, jobs, list(arrivals), max_iter, tol)
        evs = srv.stats()["evaluations"] - ev0
    lat = np.array([r["t_done"] - r["t_submit"] for r in recs])
    wait = np.array([r["t_admit"] - r["t_submit"] for r in recs])
    span = max(r["t_done"] for r in recs) - min(r["t_submit"] for r in recs)
    units = sum(n * r["report"]["iters"] for (n, _, _), r in zip(inst, recs))
    iters = [r["report"]["iters"] for r in recs]
    return {"jobs": count, "n_range": [40962, args.serve_n_hi], "precision": "mixed" if prec else "fp64",
            "grad_tol": tol, "max_iter": max_iter,
            "converged": int(sum(r["report"]["converged"] for r in recs)),
            "closed_loop_seconds": t_closed, "arrival_rate_per_s": rate, "offered_load": 0.8,
            "p50_time_to_tol_s": float(np.percentile(lat, 50)), "p99_time_to_tol_s": float(np.percentile(lat, 99)),
            "p50_queue_wait_s": float(np.percentile(wait, 50)), "makespan_s": span,
            "value": units / span, "unit": "generator-updates/s", "evaluations": evs,
            "iters_min_median_max": [int(min(iters)), int(np.median(iters)), int(max(iters))],
            "note": "jobs and N range scaled down from the 2,000-job stream for a minutes-long run"
                    if count < 2000 else None}


def run_table1(local):
    """The shape of the paper's Table 1: N = 2,562, Monte Carlo start by the
    density, the Lloyd-preconditioned LBFGS against plain LBFGS and Lloyd, with
    the paper's stopping rules (Sec. 4.1: movement 5e-4, ||g||/F <= 5e-4,
    |dF|/F < 1e-7, 2,000 iterations) and memory M = 7.  X3 and X64 (the X16
    density's formula is garbled in the paper); 7-point rule throughout."""
    import torch
    from paper_1709_06924_gb300.engine import Engine, sample_density
    out = {}
    # X64 is sampled by rho^(1/2): by rho itself all 2,562 points land inside the
    # cap (about 0.002 expected outside it), so the start has no tessellation;
    # X3 is sampled by rho as the paper states
    for name, dens, e in (("X3", I.density_x3(), 1.0), ("X64", I.density_x64(), 0.5)):
        cand, u = I.mc_candidates(400000, 2024)
        z0 = sample_density(dens, cand, u, 2562, e)
        res = {}
        for method in ("plbfgs", "lbfgs", "lloyd"):
            try:
                with Engine(2562, dens, lbfgs_m=7, device=local) as en:
                    z = torch.from_numpy(z0.copy()).cuda(local)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    r = en.lbfgs_solve(z, max_iter=2000, grad_tol=0.0, rel_grad_tol=5e-4, rel_df_tol=1e-7,
                                       step_tol=5e-4, method=method)
                    torch.cuda.synchronize()
                    t = time.perf_counter() - t0
                    cq, tq = en.mesh_quality(z)
                res[method] = {"iters": r["iters"], "fevals": r["fevals"], "seconds": t, "energy": r["energy"],
                               "grad_norm": r["grad_norm"], "status": r["status"],
                               "cellQ_min": float(cq.min()), "cellQ_mean": float(cq.mean()),
                               "triQ_min": float(tq.min()), "triQ_mean": float(tq.mean())}
            except Exception as ex:
                res[method] = {"error": repr(ex)}
        res["sampling_exponent"] = e
        out[name] = res
    return out


def run_bisection_chain(local, levels=4):
    """The paper's large-scale run (Sec. 4.3): from a converged 2,562-generator
    SCVT, bisect (every Delaunay-edge midpoint added, N -> 4N - 6) and
    optimise again, up to 655,362 generators, with the paper's stopping
    rules (movement 5e-4, ||g||/F <= 5e-4, |dF|/F < 1e-7, 2,000 iterations)
    and M = 7; FP64 form, the whole chain timed on the host clock."""
    import torch
    from paper_1709_06924_gb300.engine import Engine, sample_density
    out = {}
    for name, dens, e in (("X3", I.density_x3(), 1.0), ("X64", I.density_x64(), 0.5)):
        cand, u = I.mc_candidates(400000, 2025)
        z = torch.from_numpy(sample_density(dens, cand, u, 2562, e)).cuda(local)
        lv = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            for level in range(levels + 1):
                n = z.shape[0]
                with Engine(n, dens, lbfgs_m=7, device=local) as en:
                    tl = time.perf_counter()
                    r = en.lbfgs_solve(z, max_iter=2000, grad_tol=0.0, rel_grad_tol=5e-4, rel_df_tol=1e-7,
                                       step_tol=5e-4)
                    torch.cuda.synchronize()
                    lv.append({"n": n, "iters": r["iters"], "fevals": r["fevals"], "energy": r["energy"],
                               "grad_norm": r["grad_norm"], "seconds": time.perf_counter() - tl,
                               "status": r["status"]})
                    if level < levels:
                        z = en.bisect(z).contiguous()
            torch.cuda.synchronize()
            out[name] = {"levels": lv, "total_seconds": time.perf_counter() - t0, "sampling_exponent": e}
        except Exception as ex:
            out[name] = {"levels": lv, "error": repr(ex)}
    out["note"] = ("paper: 1296.4 s (X3) and 1914.9 s (X64) for the same chain on 128 MPI processes "
                   "(Xeon E5-2670), 4-/9-point rules; context only")
    return out


def run_ours(args, w):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_1709_06924_gb300.engine import Engine

    seed = args.seed + rank          # each replica solves its own instance
    z_host = I.uniform_sphere(w.n, seed)
    prec = 1 if args.precision == "mixed" else 0
    eng = Engine(w.n, w.density, lbfgs_m=w.lbfgs_m, device=local, precision=prec)
    z = torch.from_numpy(z_host).cuda(local)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # warm-up: W LBFGS iterations from the seeded start (history is kept);
    # then the library's autotuner picks launch shapes at the warmed iterate,
    # the state the timed steps run in (a fixed --tuning applies from the
    # start; results do not depend on either)
    if args.tuning:
        tuning = {prec: pick_tuning(args, eng, z)}
    eng.lbfgs_solve(z, max_iter=args.warmup, grad_tol=0.0)
    if not args.tuning:
        tuning = {prec: pick_tuning(args, eng, z)}
    eng.reset_stats()
    eng.set_profiling(True)
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    rep, t = timed_steps(eng, z, args.steps)
    barrier()
    clocks.stop()
    st = eng.stats()
    iters = rep["iters"]
    units, t_max = combine_ranks(w.n * iters, t, device=torch.device("cuda", local))
    value = units / t_max

    # dominant kernel, timed by CUDA events on the engine stream around each
    # launch; with concurrent cell pipelines the cell kernels overlap, so they
    # are timed on three further evaluations of the same iterate with one
    # pipeline
    quad_ms, topo_ms, stq = one_pipeline_kernel_ms(eng, z)
    roofline = roofline_of(prec, w, quad_ms, topo_ms, stq, tuning[prec]["topo_cell_lanes"])

    # end to end through the C ABI with host buffers: a second engine replays
    # the same warm-up (evaluations are deterministic, so it reaches the same
    # state), then the same K iterations run with Z in pinned host memory:
    # every step copies Z in, checks it against the engine's iterate, runs one
    # iteration and copies the result back
    e2e = None
    if not args.no_e2e:
        eng2 = Engine(w.n, w.density, lbfgs_m=w.lbfgs_m, device=local, precision=prec)
        eng2.set_tuning(**tuning[prec])
        z2 = torch.from_numpy(z_host).cuda(local)
        eng2.lbfgs_solve(z2, max_iter=args.warmup, grad_tol=0.0)
        zp = torch.empty((w.n, 3), dtype=torch.float64, pin_memory=True)
        zp.copy_(z2.cpu())
        del z2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(eng2.stream)
        k_e2e = 0
        for _ in range(args.steps):
            r = eng2.lbfgs_solve(zp.numpy(), max_iter=1, grad_tol=0.0, warm_start=2)
            k_e2e += r["iters"]
        e1.record(eng2.stream)
        torch.cuda.synchronize()
        te = e0.elapsed_time(e1) / 1e3
        same = bool(np.array_equal(zp.numpy(), z.cpu().numpy()))
        eng2.close()
        ue, te = combine_ranks(w.n * k_e2e, te, device=torch.device("cuda", local))
        e2e = {"value": ue / te, "unit": "generator-updates/s",
               "h2d_bytes_per_step": w.n * 24, "d2h_bytes_per_step": w.n * 24,
               "same_iterates_as_device_run": same}

    # the other precision form on the same workload, same W and K
    other = None
    if not args.no_other_form:
        oprec = 1 - prec
        eng3 = Engine(w.n, w.density, lbfgs_m=w.lbfgs_m, device=local, precision=oprec)
        z3 = torch.from_numpy(z_host).cuda(local)
        if args.tuning:
            tuning[oprec] = pick_tuning(args, eng3, z3)
        eng3.lbfgs_solve(z3, max_iter=args.warmup, grad_tol=0.0)
        if not args.tuning:
            tuning[oprec] = pick_tuning(args, eng3, z3)
        eng3.reset_stats()
        eng3.set_profiling(True)
        torch.cuda.synchronize()
        rep3, t3 = timed_steps(eng3, z3, args.steps)
        st3 = eng3.stats()
        q3, tp3, stq3 = one_pipeline_kernel_ms(eng3, z3)
        eng3.close()
        u3, t3 = combine_ranks(w.n * rep3["iters"], t3, device=torch.device("cuda", local))
        other = {"precision": "mixed" if oprec else "fp64", "dtype": "f32/f64" if oprec else "f64+f32x2",
                 "value": u3 / t3, "ms_per_step": 1e3 * t3 / max(rep3["iters"], 1),
                 "roofline": roofline_of(oprec, w, q3, tp3, stq3, tuning[oprec]["topo_cell_lanes"]),
                 "eval_ms_avg": st3["eval_ms"] / max(st3["evaluations"], 1), "tuning": tuning[oprec]}

    batched = None
    if not args.no_batched:
        try:
            batched = {"fp64": run_batched(args, local, 0), "mixed": run_batched(args, local, 1)}
        except Exception as ex:  # reported, not fatal to the headline line
            batched = {"error": repr(ex)}

    serving = None
    if not args.no_serving:
        try:
            serving = run_serving(args, local, prec)
        except Exception as ex:  # reported, not fatal to the headline line
            serving = {"error": repr(ex)}

    table1 = None
    if not args.no_table1:
        try:
            table1 = run_table1(local)
        except Exception as ex:  # reported, not fatal to the headline line
            table1 = {"error": repr(ex)}

    chain = None
    if not args.no_chain:
        try:
            chain = run_bisection_chain(local)
        except Exception as ex:  # reported, not fatal to the headline line
            chain = {"error": repr(ex)}

    ttt = None
    if not args.no_time_to_tol:
        for pr in (0, 1):
            if pr not in tuning:
                with Engine(w.n, w.density, lbfgs_m=w.lbfgs_m, device=local, precision=pr) as et:
                    zt_ = torch.from_numpy(z_host).cuda(local)
                    tuning[pr] = pick_tuning(args, et, zt_)
        ttt = {"fp64": time_to_tolerance(w, z_host, local, 0, tuning[0]),
               "mixed": time_to_tolerance(w, z_host, local, 1, tuning[1])}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w, args.cpu_sample_n, args.cpu_sample_iters, args.seed)

    if rank == 0:
        line = {
            "metric": "generator-updates/s", "value": value, "unit": "generator-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / max(iters, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64" if prec else "f64+f32x2", "data": "synthetic",
            "config": {"workload": w.name, "n_generators": w.n, "density": "tanh cap",
                       "gamma": w.density.gamma, "alpha": w.density.alpha, "beta": w.density.beta,
                       "lbfgs_m": w.lbfgs_m, "quadrature": "7-point per sub-triangle", "seed": args.seed,
                       "precision": args.precision, "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "inputs larger than L2 (history %d MB per step)" % (2 * w.lbfgs_m * w.n * 24 >> 20),
                       "iters_timed": iters, "fevals_timed": rep["fevals"], "tuning": tuning[prec]},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks.summary(),
            "gpu_launches": st["kernel_launches"],
            "other_form": other,
            "time_to_tol": ttt,
            "batched": batched,
            "serving": serving,
            "paper_table1": table1,
            "bisection_chain": chain,
            "knn_retries": st["knn_retries"],
            "ambiguous": st["ambiguous"],
            "eval_ms_avg": st["eval_ms"] / max(st["evaluations"], 1),
            "lbfgs_ms_total": st["lbfgs_ms"],
            "fevals_per_s": st["evaluations"] / t_max if t_max > 0 else None,
            "roofline_two_loop": two_loop_roofline(w, args.warmup, iters, st["lbfgs_ms"]),
        }
        print(json.dumps(line), flush=True)
    eng.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


# FP64 exp per call in DFMA equivalents (measured like the other per-call costs)
EXP_DFMA = 17.9


def fp64_flops_per_generator(kind: int, series_frac: float = 0.0, series_len: float = 0.0) -> float:
    """FP64 work of the quadrature kernel per generator, in flop equivalents.

    Per Voronoi edge the method integrates two signed sub-triangles (Sec.
    3.2.2): per sub-triangle the Van Oosterom-Strackee area (differences,
    cross and dot products: 38 flops, one atan2) and 7 rule points; per point
    the projected point (combination, norm, rsqrt, scale: 37 + rsqrt), the
    density, the weight and the accumulation of m, c and |p - z|^2 (24).  The
    tanh cap evaluated directly costs a cross product, a norm and a dot (19),
    sqrt, atan2, exp and a division (its logistic form) (+5); from the
    cell's Taylor series it costs a dot, a difference and a Horner sweep of
    series_len terms (6 + 2 series_len), for the fraction series_frac of the
    cells that use one (the series themselves are built by a separate
    kernel).  X3 costs 6.  A transcendental is charged what it costs on this
    GPU in FMA-pipe time (per-call costs measured with CUDA events, in DFMA
    equivalents x 2 flop).  The cell of a generator has 6 edges on average
    (Euler: 2E = 6N - 12).
    """
    rsqrt, sqrt, atan2, exp, div = 2 * 6.9, 2 * 9.6, 2 * 41.0, 2 * EXP_DFMA, 2 * 10.4
    direct = {0: 0.0, 1: 6.0, 2: 24.0 + sqrt + atan2 + exp + div, 3: 28.0 + sqrt + atan2 + exp + div}[kind]
    dens = direct
    if kind >= 2:
        dens = series_frac * (6.0 + 2.0 * series_len) + (1.0 - series_frac) * direct
    point = 37.0 + rsqrt + 24.0 + dens
    subtri = 38.0 + atan2 + 7 * point
    mu = 11.0 + rsqrt
    return 6.0 * (2 * subtri + mu)


def measured_hbm_gbs():
    """HBM copy bandwidth measured on this machine (MEASURED_PEAKS.json), else
    the fallback figure."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def two_loop_roofline(w, warmup, iters, lbfgs_ms):
    """HBM roofline of the two-loop recursion (Sec. 2.2.2 with diag(h) as the
    initial inverse Hessian): algorithmic traffic per generator (4c + 2) x 24
    bytes with c stored pairs (each history vector read twice, g read, q
    written), c = min(warm-up + i, m) in timed iteration i, over the CUDA-event
    time of the two-loop launches in the timed steps.  The fused kernels read
    and write q once per pair step, 72 + 192 c bytes per generator."""
    if not iters or lbfgs_ms <= 0:
        return None
    counts = [min(warmup + i, w.lbfgs_m) for i in range(iters)]
    alg = sum((4 * c + 2) * 24 for c in counts) * w.n
    impl = sum(72 + 192 * c for c in counts) * w.n
    peak, src = measured_hbm_gbs()
    achieved = alg / (lbfgs_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "two-loop (k_neg, k_axpy, k_finish_scalar)", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
            "algorithmic_bytes": alg, "implementation_bytes": impl,
            "implementation_gbs": impl / (lbfgs_ms * 1e-3) / 1e9, "peak_source": src, "pairs_per_iteration": counts}


def fp64_peak_tflops() -> float:
    return 152 * 2 * 2 * 2.07e9 / 1e12


# Instruction issue is what bounds the double-float quadrature and the
# topology pass: each of the 152 SMs' four schedulers issues at most one warp
# instruction per clock (2.07 GHz), 1.2586e12 warp instructions per second.
# The work per unit is the instruction count ncu measured (one-pass
# smsp__inst_executed.sum) for a launch of the timed steps of this bench at
# N = 2,621,442, divided by N (profiles/launches_tanh_2621442.md); the
# topology pass's count depends on its lanes per cell.
ISSUE_PEAK = 152 * 4 * 2.07e9
QUAD_INST_PER_GENERATOR = 4536632457 / 2621442
TOPO_INST_PER_CELL = {32: 3153936979 / 2621442, 16: 1873542833 / 2621442}


def one_pipeline_kernel_ms(eng, z, evals=3):
    """Average CUDA-event time of the quadrature and of the first topology
    pass over `evals` evaluations of z with one cell pipeline (the engine's
    tuning is restored afterwards; stats are reset)."""
    tsave = eng.tuning()
    eng.set_tuning(**dict(tsave, chunks=1))
    eng.set_profiling(True)
    eng.evaluate(z)
    eng.reset_stats()
    for _ in range(evals):
        eng.evaluate(z)
    st = eng.stats()
    eng.set_tuning(**tsave)
    quad = st["cell_kernel_ms"] / max(st["cell_kernel_timed"], 1)
    topo = st["topo_kernel_ms"] / max(st["topo_kernel_timed"], 1)
    return quad, topo, st


def roofline_of(prec, w, quad_ms, topo_ms, st, lanes=32):
    """Roofline of the step's dominant kernel: the double-float quadrature in
    the FP64 form, the topology pass in the mixed form; both issue-bound."""
    if prec == 0:
        sfrac = st["series_cells"] / max(w.n * st["evaluations"], 1)
        slen = st["series_terms"] / max(st["series_cells"], 1)
        flops_gen = fp64_flops_per_generator(w.density.kind, sfrac, slen)
        achieved = w.n * QUAD_INST_PER_GENERATOR / (quad_ms * 1e-3) / 1e12
        return {"bound": "alu", "kernel": "k_quad", "achieved": achieved, "peak": ISSUE_PEAK / 1e12,
                "unit": "Twarp-inst/s", "frac": achieved * 1e12 / ISSUE_PEAK, "traffic": quad_traffic_bytes(w.n),
                "avg_launch_ms": quad_ms, "inst_per_generator": QUAD_INST_PER_GENERATOR,
                "fp64_equivalent_tflops": w.n * flops_gen / (quad_ms * 1e-3) / 1e12,
                "fp64_flop_equivalents_per_generator": flops_gen,
                "fp64_pipe_peak_tflops": fp64_peak_tflops(),
                "series_cell_fraction": sfrac, "series_terms_avg": slen,
                "peak_source": "instruction issue: 152 SMs x 4 schedulers x 1 warp-instruction/clk x 2.07 GHz",
                "work_source": "ncu smsp__inst_executed.sum of a k_quad launch of the timed steps at "
                               "N = 2,621,442, per generator (double-float arithmetic: FP32 pairs, FP64 for "
                               "per-edge offsets)",
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_quad launch "
                                  "at N = 163,842, scaled by N (profiles/k_quad_tanh_163842.md)"}
    ipc = TOPO_INST_PER_CELL[lanes]
    achieved = w.n * ipc / (topo_ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "k_topo_warp", "achieved": achieved, "peak": ISSUE_PEAK / 1e12,
            "unit": "Twarp-inst/s", "frac": achieved * 1e12 / ISSUE_PEAK, "traffic": None,
            "avg_launch_ms": topo_ms, "quad_kernel_ms": quad_ms, "inst_per_cell": ipc, "lanes_per_cell": lanes,
            "peak_source": "instruction issue: 152 SMs x 4 schedulers x 1 warp-instruction/clk x 2.07 GHz",
            "work_source": "ncu smsp__inst_executed.sum of a k_topo_warp launch of the timed steps at "
                           "N = 2,621,442, per cell"}


def quad_traffic_bytes(n: int):
    """DRAM bytes of one k_quad launch: ncu at N = 163,842 (118.31 MB read +
    19.11 MB written, tanh cap, density series on), scaled by the number of
    generators."""
    return (118.309376e6 + 19.114240e6) * n / 163842


def main():
    args = parse()
    w = I.WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
