#!/usr/bin/env python
"""Benchmark: explicit finite-volume sweep on GB300 (arXiv 2209.13768, Sec. 3.1).

Default workload: one 512^3 grid, fp32 field, per-cell conductivity
k ~ lognormal(0, 0.5), x faces Dirichlet 1 / 0, y and z zero-flux,
dt = 0.9 x the stability limit; one benchmark step = one 1000-step solve
(every time step of the sweep, fused `depth` steps per pass over the grid).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. `value` is cell-updates/s (in GLUPS) with the inputs
resident in HBM (device-side CUDA events, max over ranks); `e2e` is the same
metric through the C ABI from pinned host buffers (field and conductivity in,
result out, copies inside the timed region). Multi-GPU runs are independent
replicas (weak scaling): the sweep of one grid is a single-GPU problem here.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s (GLUPS) and % HBM roofline on 1 GB300; serving p50/p99 latency"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
KERNEL_SOURCES = ["paper_2209_13768_gb300/csrc/wfa_sweep_col.cuh", "paper_2209_13768_gb300/csrc/wfa_sweep.cuh",
                  "paper_2209_13768_gb300/csrc/wfa_internal.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["lognormal", "heat64", "advdiff", "advdiff_bf16", "batch", "serve",
                                           "implicit", "implicit_lognormal", "dsl_heat"],
                    default="lognormal")
    ap.add_argument("--rtol", type=float, default=1e-6, help="implicit: CG tolerance ||r|| <= rtol ||b||")
    ap.add_argument("--cg", choices=["classic", "pipelined"], default="classic",
                    help="implicit: classic CG or Chronopoulos-Gear (one reduction an iteration)")
    ap.add_argument("--serve-requests", type=int, default=10000,
                    help="requests of the serving stream added to the line (0: none; 10^4 at 200/s is 50 s)")
    ap.add_argument("--solve-steps", type=int, default=0, help="time steps per benchmark step (0: workload default)")
    ap.add_argument("--shape", type=str, default="", help="NX,NY,NZ: same physics on another grid (profiling)")
    ap.add_argument("--depth", type=int, default=0, help="fused steps per pass (0: tuned)")
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-solo", action="store_true", help="batch: skip the one-grid-per-launch comparison")
    ap.add_argument("--zchunk", type=int, default=0, help="planes per z chunk of the column kernels (0: tuned)")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the oracle comparison of the bench line")
    ap.add_argument("--split", choices=["none", "z"], default="none",
                    help="z: one grid split into slabs along z, one slab per rank (NCCL plane exchange "
                         "before every step), or --slabs slabs on one GPU")
    ap.add_argument("--slabs", type=int, default=0, help="--split z on one GPU: number of slabs (default 2)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line: skip the advection-diffusion and batch configurations")
    return ap.parse_args()


def max_over_ranks(x, dist, device):
    """Largest x over all ranks: the slowest replica sets the job's time."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, updates_per_rank, seconds):
    """Whole-job GLUPS: every rank advances its own replica (weak scaling)."""
    return world * updates_per_rank / seconds / 1e9


DEVICE_MATH_MARK = b"// ----------------------------------------------------------- device math --"


def kernel_hash():
    """Hash of the sweep kernels' device code: their own headers, plus the
    device-math part of wfa_internal.cuh (its host declarations above the
    marker do not change the kernels)."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            text = f.read()
        if rel.endswith("wfa_internal.cuh") and DEVICE_MATH_MARK in text:
            text = text[text.index(DEVICE_MATH_MARK):]
        h.update(text)
    return h.hexdigest()[:16]


def workload(name, solve_steps, shape=""):
    from paper_2209_13768_gb300 import workloads as W
    kw = {"shape": tuple(int(v) for v in shape.split(","))} if shape else {}
    if name == "lognormal":
        p = W.heat_lognormal(**kw)
    elif name == "heat64":
        p = W.heat_64()
    else:
        p = W.advection_diffusion(**kw)
    if solve_steps:
        p.steps = solve_steps
    return p


def bytes_per_cell(storage_bf16, kvar):
    """Algorithmic HBM bytes per cell per pass: read + write of the field,
    plus one read of k (Eq. A_eff = 2 D_u + D_k)."""
    e = 2 if storage_bf16 else 4
    return 2 * e + (4 if kvar else 0)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_rate(p, budget_s):
    """The oracle as it stands, on this host's cores, on a bounded sample of
    the workload (a few time steps of the same grid)."""
    import numpy as np

    import oracle
    k = p.k if isinstance(p.k, float) else np.asarray(p.k, dtype=np.float64)
    dt = p.dt if p.dt else 0.9 * oracle.dt_max(shape=p.shape, h=p.h, k=k, u=p.u, bc=p.bc)
    T = np.asarray(p.T0, dtype=np.float64)
    cells = p.shape[0] * p.shape[1] * p.shape[2]
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()   # one core: a single time step of the grid
    T = oracle.run(T, 1, shape=p.shape, h=p.h, k=k, u=p.u, bc=p.bc, dt=dt, threads=1)
    el1 = time.perf_counter() - t0
    t0 = time.perf_counter()   # then every core (warm-up step)
    T = oracle.run(T, 1, shape=p.shape, h=p.h, k=k, u=p.u, bc=p.bc, dt=dt, threads=cores)
    one = time.perf_counter() - t0
    n = max(1, min(50, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(T, n, shape=p.shape, h=p.h, k=k, u=p.u, bc=p.bc, dt=dt, threads=cores)
    el = time.perf_counter() - t0
    return {"value": cells * n / el / 1e9, "unit": "GLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{n} fp64 time steps of the {p.shape[0]}x{p.shape[1]}x{p.shape[2]} grid "
                      f"({p.name}), OpenMP over all host cores, after 1 warm-up step",
            "value_1_core": cells / el1 / 1e9, "sample_1_core": "one fp64 time step of the same grid on one core"}


def reference_arm(args, rank):
    """--impl reference: the FP64 oracle on the host cores, same metric/config."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    if args.workload in ("implicit", "implicit_lognormal"):
        from paper_2209_13768_gb300 import workloads as W
        shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else W.IMPLICIT_SHAPE
        p = W.implicit_problem(shape, lognormal=args.workload == "implicit_lognormal")
        kk = p.k if np.isscalar(p.k) else np.asarray(p.k, dtype=np.float64)
        cells = shape[0] * shape[1] * shape[2]
        per_step = 2   # each benchmark step: one time step of two CG iterations on the full grid
        run = lambda: oracle.implicit(p.T0, 1, shape=p.shape, h=p.h, k=kk, bc=p.bc, dt=p.dt, rtol=0.0,
                                      max_iter=per_step)
        for _ in range(args.warmup):
            run()
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            run()
            times.append(time.perf_counter() - t0)
        total = sum(times)
        value = cells * per_step * args.steps / total / 1e9
        unit = "G cell-iterations/s"
        line = {"impl": "reference", "metric": "CG cell-iterations/s (G) of the implicit step, and % HBM roofline "
                "on 1 GB300", "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": p.name, "cells": cells,
                           "sample": f"one time step of {per_step} CG iterations per benchmark step"},
                "cpu_baseline": {"value": value, "unit": unit, "cores": os.cpu_count(), "kind": "oracle",
                                 "sample": f"one fp64 time step of {per_step} CG iterations (set-up included)"},
                "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    p = workload(args.workload, args.solve_steps, args.shape)
    k = p.k if isinstance(p.k, float) else np.asarray(p.k, dtype=np.float64)
    dt = p.dt if p.dt else 0.9 * oracle.dt_max(shape=p.shape, h=p.h, k=k, u=p.u, bc=p.bc)
    T = np.asarray(p.T0, dtype=np.float64)
    cells = p.shape[0] * p.shape[1] * p.shape[2]
    per_step = 1   # each benchmark step: one time step of the grid (bounded sample)
    for _ in range(args.warmup):
        T = oracle.run(T, per_step, shape=p.shape, h=p.h, k=k, u=p.u, bc=p.bc, dt=dt)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        T = oracle.run(T, per_step, shape=p.shape, h=p.h, k=k, u=p.u, bc=p.bc, dt=dt)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = cells * per_step * args.steps / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": p.name, "cells": cells, "sample": f"{per_step} time step per benchmark step"},
            "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{per_step} fp64 time step of the full grid per benchmark step"},
            "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _pct(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, int(q * (len(v) - 1) + 0.5))] if v else None


def serving_sample(n_requests, rate=200.0, seed=5, quantum=64, fifo_requests=1000, lookahead=192):
    """The serving configuration: Poisson arrivals (rate per second) of heat /
    advection-diffusion solves, each with its own shape (edges log-uniform in
    [32, 256]) and its own fields, steps U{50..2000}, fp32 or bf16, through the
    continuous-batching server (HBM budget 120 GB); then the first
    fifo_requests arrivals of the same stream through the plain form (one grid
    at a time, first come first served, wfa_step). Worker threads generate each
    request's fields ahead of its arrival (at most `lookahead` in host memory).
    Latency: from the scheduled arrival to the result on the host (the
    server's submit-to-result time plus how late the submit was)."""
    import concurrent.futures as cf
    import threading

    import paper_2209_13768_gb300 as wfa
    from paper_2209_13768_gb300 import workloads as W
    specs = W.request_specs(rate=rate, count=n_requests, seed=seed)
    cells = [s.shape[0] * s.shape[1] * s.shape[2] for s in specs]
    updates = [c * s.steps for c, s in zip(cells, specs)]

    def stream(count):
        """(spec, problem) in arrival order, generated ahead by a thread pool."""
        with cf.ThreadPoolExecutor(8) as ex:
            futs = {}
            for i in range(min(lookahead, count)):
                futs[i] = ex.submit(W.make_request, specs[i])
            for i in range(count):
                p = futs.pop(i).result()
                if i + lookahead < count:
                    futs[i + lookahead] = ex.submit(W.make_request, specs[i + lookahead])
                yield specs[i], p

    def run_server():
        late, lat = [], [None] * n_requests
        pending = []                  # (index, ticket, lateness) not yet collected
        lock = threading.Lock()
        stop = threading.Event()
        with wfa.Server(budget_bytes=120 << 30, quantum=quantum) as srv:

            def collect():            # latencies of finished tickets, freeing their arrays
                while True:
                    with lock:
                        items = list(pending)
                    left = []
                    for i, tk, lt in items:
                        if srv.poll(tk) == 1:
                            lat[i] = srv.latency(tk) + lt
                            srv.wait(tk, timeout=1.0)
                        else:
                            left.append((i, tk, lt))
                    with lock:
                        done = {i for i, _, _ in items} - {i for i, _, _ in left}
                        pending[:] = [e for e in pending if e[0] not in done]
                        empty = not pending
                    if stop.is_set() and empty:
                        return
                    time.sleep(0.002)

            th = threading.Thread(target=collect)
            th.start()
            t0 = time.perf_counter()
            for i, (spec, p) in enumerate(stream(n_requests)):
                wait = spec.t - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
                lateness = max(0.0, time.perf_counter() - t0 - spec.t)
                tk = srv.submit(p.shape, p.T0, spec.steps, h=p.h, storage=spec.storage, k=p.k, u=p.u, bc=p.bc,
                                dt=p.dt)
                late.append(lateness)
                with lock:
                    pending.append((i, tk, lateness))
            stop.set()
            th.join()
            wall = time.perf_counter() - t0
            st = srv.stats()
        return wall, lat, late, st

    def run_fifo(count):
        lat = []
        t0 = time.perf_counter()
        for spec, p in stream(count):
            wait = spec.t - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            with wfa.Grid(p.shape, h=p.h, storage=spec.storage) as g:
                g.set_bcs(p.bc)
                g.set_coeffs(p.k, p.u)
                g.set_field(p.T0)
                g.set_dt(p.dt if p.dt else 0.9 * g.stability_dt())
                g.step(spec.steps)
                g.read_field()
            lat.append(time.perf_counter() - t0 - spec.t)
        return time.perf_counter() - t0, lat

    wall_s, lat_s, late, st = run_server()
    nf = min(fifo_requests, n_requests)
    wall_f, lat_f = run_fifo(nf)
    thirds = [lat_s[i * n_requests // 3:(i + 1) * n_requests // 3] for i in range(3)]
    span = specs[-1].t
    return {"requests": n_requests, "rate_per_s": rate, "arrival_span_s": span,
            "offered_GLUPS": sum(updates) / span / 1e9,
            "inputs": "every request its own shape and fields (seeded), generated ahead of its arrival",
            "continuous_batching": {
                "GLUPS": sum(updates) / wall_s / 1e9, "wall_s": wall_s, "p50_s": _pct(lat_s, 0.5),
                "p99_s": _pct(lat_s, 0.99), "p99_s_by_third_of_stream": [_pct(t, 0.99) for t in thirds],
                "p50_s_by_third_of_stream": [_pct(t, 0.5) for t in thirds], "ticks": st["ticks"],
                "gpu_busy_s": st["busy_seconds"], "peak_resident_GB": st["peak_resident_bytes"] / 1e9,
                "max_submit_lateness_s": max(late) if late else 0.0},
            "one_grid_per_launch_fifo": {
                "requests": nf, "GLUPS": sum(updates[:nf]) / wall_f / 1e9, "wall_s": wall_f,
                "p50_s": _pct(lat_f, 0.5), "p99_s": _pct(lat_f, 0.99),
                "stream": f"the first {nf} arrivals of the same stream"}}


def batch_bench(args, emit=True):
    """256 grids, edges log-uniform in [16,128], k lognormal(0,0.5), steps
    U{50..500}: one persistent CUDA-graph launch vs one grid at a
    time through wfa_step."""
    import numpy as np
    import torch

    import paper_2209_13768_gb300 as wfa
    from paper_2209_13768_gb300 import workloads as W
    probs = W.batch_grids()
    grids = []
    for p in probs:
        g = wfa.Grid(p.shape)
        g.set_bcs(p.bc)
        g.set_coeffs(p.k, p.u)
        g.set_field(p.T0)
        g.set_dt(0.9 * g.stability_dt())
        grids.append(g)
    steps = [p.steps for p in probs]
    cells = [p.shape[0] * p.shape[1] * p.shape[2] for p in probs]
    updates = sum(c * n for c, n in zip(cells, steps))
    wfa.batch_run(grids, [1] * len(grids))   # builds the graph
    for _ in range(args.warmup):
        wfa.batch_run(grids, steps)
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.synchronize()
    sampler.start()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        wfa.batch_run(grids, steps)   # returns when the work is done
        times.append(time.perf_counter() - t0)
    clocks = sampler.stop()
    t_batch = sum(times) / args.steps
    t_solo = float("nan")
    if not args.no_solo:
        for g, n in zip(grids, steps):   # warm-up: graphs of the small grids, tuned kernels
            g.step(n)
        for g in grids:
            g.sync()
        t0 = time.perf_counter()
        for g, n in zip(grids, steps):
            g.step(n)
        for g in grids:
            g.sync()
        t_solo = time.perf_counter() - t0
    for g in grids:
        g.close()
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = bytes_per_cell(False, True) * updates / t_batch / 1e9
    line = {"metric": METRIC, "value": updates / t_batch / 1e9, "unit": "GLUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_batch, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "256 grids, edges log-uniform [16,128], k lognormal(0,0.5), steps U{50..500}",
                       "grids": len(probs), "cells": sum(cells), "cell_updates_per_step": updates,
                       "timing": "host wall clock around wfa_batch_run (one graph launch, waits for the work)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "bytes_per_cell_update": 12,
                         "scope": "the whole batched call (every kernel of every round, the graph launch)"},
            "one_grid_per_launch": None if args.no_solo else
            {"value": updates / t_solo / 1e9, "unit": "GLUPS", "ms_per_step": 1e3 * t_solo,
             "form": "wfa_step on each grid in turn (its own tuned kernels and step graphs), one stream"},
            "gpu_launches": None, "clocks": clocks}
    if emit:
        print(json.dumps(line), flush=True)
    return line


CG_SOURCES = ["paper_2209_13768_gb300/csrc/wfa_implicit.cu"]


def cg_kernel_hash():
    h = hashlib.sha256()
    for rel in CG_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def cg_bytes_per_cell(kvar):
    """Algorithmic HBM bytes per cell per CG iteration: cg_spmv reads r and
    p_old and writes p and q (16 B, + 4 B of 1/k for per-cell k); cg_update
    reads x, p, q, r and writes x, r (24 B). The pipelined kernel moves the
    same 40 B (+4): reads r, w, s, p, x, writes them."""
    return 40 + (4 if kvar else 0)


def implicit_bench(args, rank, world, dist):
    """Backward-Euler steps solved by classic CG (Sec. 1.1.2, Eq. impl_form):
    512^3, omega = 1/10, held boundary layers; a benchmark step is
    --solve-steps time steps (default 10), each CG to --rtol."""
    import numpy as np
    import torch

    import paper_2209_13768_gb300 as wfa
    from paper_2209_13768_gb300 import workloads as W
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else W.IMPLICIT_SHAPE
    p = W.implicit_problem(shape, steps=args.solve_steps or 10, lognormal=args.workload == "implicit_lognormal")
    kvar = not np.isscalar(p.k)
    cells = shape[0] * shape[1] * shape[2]
    stream = torch.cuda.Stream()
    g = wfa.Grid(p.shape, h=p.h, stream=stream.cuda_stream)
    g.set_bcs(p.bc)
    g.set_coeffs(p.k)
    g.set_field(p.T0)
    g.set_cg_method(args.cg)
    max_iter = 1000
    for _ in range(args.warmup):
        g.implicit_step(p.dt, p.steps, rtol=args.rtol, max_iter=max_iter)
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = g.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    iters = 0
    res = 0.0
    for i in range(args.steps):
        ev[i][0].record(stream)
        it, res = g.implicit_step(p.dt, p.steps, rtol=args.rtol, max_iter=max_iter)
        ev[i][1].record(stream)
        iters += it
    torch.cuda.synchronize()
    clocks = sampler.stop()
    gpu_launches = g.launch_count() - launches0
    total_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    total_s = max_over_ranks(total_s, dist, "cuda")
    value = world * cells * iters / total_s / 1e9
    bpc = cg_bytes_per_cell(kvar)
    achieved = bpc * cells * iters / total_s / 1e9
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    traffic = None   # DRAM bytes of one CG iteration (cg_spmv + cg_update) from ncu, if current
    try:
        with open(TRAFFIC_FILE) as f:
            ent = json.load(f).get(f"implicit:{'k' if kvar else 'u'}:cg_iteration")
        if ent and ent.get("kernel_hash") == cg_kernel_hash() and shape == W.IMPLICIT_SHAPE and args.cg == "classic":
            traffic = ent["bytes_per_iteration"]
    except (OSError, ValueError):
        pass
    e2e = None
    if not args.no_e2e:
        T0h = torch.from_numpy(np.ascontiguousarray(p.T0)).pin_memory()
        outh = torch.empty(tuple(p.T0.shape), dtype=torch.float32).pin_memory()
        e2e_t, e2e_it = [], 0
        for i in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.set_field(T0h)
            it, _ = g.implicit_step(p.dt, p.steps, rtol=args.rtol, max_iter=max_iter)
            g.read_field(outh)
            if i:
                e2e_t.append(time.perf_counter() - t0)
                e2e_it += it
        e2e_s = max_over_ranks(sum(e2e_t), dist, "cuda")
        e2e = {"value": world * cells * e2e_it / e2e_s / 1e9, "unit": "G cell-iterations/s",
               "h2d_bytes_per_step": cells * 4, "d2h_bytes_per_step": cells * 4,
               "ms_per_step": 1e3 * e2e_s / len(e2e_t)}
    g.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        kk = p.k if np.isscalar(p.k) else np.asarray(p.k, dtype=np.float64)
        t0 = time.perf_counter()
        oracle.implicit(p.T0, 1, shape=p.shape, h=p.h, k=kk, bc=p.bc, dt=p.dt, rtol=0.0, max_iter=1)
        one = time.perf_counter() - t0
        m = max(1, min(50, int(args.cpu_seconds / max(one, 1e-6))))
        t0 = time.perf_counter()
        oracle.implicit(p.T0, 1, shape=p.shape, h=p.h, k=kk, bc=p.bc, dt=p.dt, rtol=0.0, max_iter=m)
        el = time.perf_counter() - t0
        cpu = {"value": cells * m / el / 1e9, "unit": "G cell-iterations/s", "cores": os.cpu_count(),
               "kind": "oracle", "sample": f"one fp64 time step of {m} CG iterations on the full grid "
                                           "(set-up and the initial residual included), OpenMP face passes"}
    if rank == 0:
        line = {"metric": "CG cell-iterations/s (G) of the implicit step, and % HBM roofline on 1 GB300",
                "value": value, "unit": "G cell-iterations/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": p.name, "cells": cells, "time_steps_per_step": p.steps, "dt": p.dt,
                           "omega": p.dt, "rtol": args.rtol, "cg": args.cg, "cg_iterations": iters,
                           "cg_iterations_per_time_step": iters / (p.steps * args.steps), "last_rel_residual": res,
                           "conductivity": "per-cell lognormal(0,0.5)" if kvar else "uniform 1",
                           "l2": "inputs larger than L2 (six 512 MiB vectors)", "parallelism": f"replicas x{world}"},
                "cg_iterations_per_s": world * iters / total_s,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per CG iteration",
                             "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                             "bytes_per_cell_per_iteration": bpc, "frac_of_nominal_8TBps": achieved / 8000.0,
                             "scope": "the whole solve: every kernel of the timed steps (cg_init, cg_spmv, "
                                      "cg_update and the loop-control kernels; pipelined: cg_init, cg_spmv once a "
                                      "step, cg_pipe), one graph launch a call"},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches, "clocks": clocks}
        print(json.dumps(line), flush=True)


def dsl_bench(args, rank, world, dist):
    """The expression front end on the paper's explicit heat update
    (Eq. expl_form, omega = 1/10, held boundary cells), 512^3 fp32: the
    generated kernel against the same physics through wfa_step."""
    import numpy as np
    import torch

    import paper_2209_13768_gb300 as wfa
    from paper_2209_13768_gb300 import stencil as S
    from paper_2209_13768_gb300 import workloads as W
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else (512, 512, 512)
    nx, ny, nz = shape
    T, w = S.Field("T"), S.Param("w")
    step = S.compile({T: T + w * (T[-1, 0, 0] + T[1, 0, 0] + T[0, -1, 0] + T[0, 1, 0] + T[0, 0, -1] + T[0, 0, 1]
                                  - 6 * T)})
    T0 = W.uniform01(shape, 3)
    for a in range(3):   # held layers at 0
        idx = [slice(None)] * 3
        idx[2 - a] = 0
        T0[tuple(idx)] = 0.0
        idx[2 - a] = -1
        T0[tuple(idx)] = 0.0
    steps = args.solve_steps or 200
    t = torch.tensor(T0, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step.run({"T": t}, steps=steps, w=0.1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    n0 = step.launches
    torch.cuda.synchronize()
    for i in range(args.steps):
        ev[i][0].record(stream)
        step.run({"T": t}, steps=steps, w=0.1)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    total_s = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, dist, "cuda")
    cells = nx * ny * nz
    value = world * cells * steps * args.steps / total_s / 1e9
    # the hand-written path on the same physics (held layers on every face)
    with wfa.Grid(shape) as g:
        g.set_bcs([("dirichlet_cell", 0.0)] * 6)
        g.set_coeffs(1.0)
        g.set_field(T0)
        g.set_dt(0.1)
        g.step(steps)
        g.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(steps * args.steps)
        g.sync()
        hand = cells * steps * args.steps / (time.perf_counter() - t0) / 1e9
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = 8 * cells * steps * args.steps / total_s / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": "cell-updates/s (GLUPS) of the generated stencil kernel, and % HBM roofline on 1 GB300",
            "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"expression front end: heat, omega = 0.1, held layers, {nx}x{ny}x{nz}",
                       "time_steps_per_step": steps, "l2": "inputs larger than L2 (512 MiB field)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "bytes_per_cell": 8},
            "hand_written_wfa_step_GLUPS": hand, "gpu_launches": step.launches - n0}), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2209_13768_gb300 as wfa
    from paper_2209_13768_gb300 import build as wfa_build
    wfa_build.build()
    if args.workload == "batch":
        batch_bench(args)
        return
    if args.workload == "serve":
        print(json.dumps({"metric": METRIC, "serving": serving_sample(args.serve_requests or 400)}), flush=True)
        return
    if args.workload in ("implicit", "implicit_lognormal"):
        implicit_bench(args, rank, world, dist)
        return
    if args.workload == "dsl_heat":
        dsl_bench(args, rank, world, dist)
        return
    if args.split == "z":
        split_bench(args, rank, world, dist, local)
        return

    p = workload(args.workload, args.solve_steps, args.shape)
    storage = wfa.BF16 if args.workload == "advdiff_bf16" else wfa.F32
    r = grid_bench(args, p, storage, world, rank, dist, local, e2e=not args.no_e2e,
                   accuracy=not args.no_accuracy)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_rate(p, args.cpu_seconds)
    default = args.workload == "lognormal" and not args.shape and not args.solve_steps
    serving = None
    if rank == 0 and world == 1 and args.serve_requests and default:
        serving = serving_sample(args.serve_requests)
    extras = {}
    if rank == 0 and world == 1 and default and not args.no_extras:
        # the other single-GPU configurations, driver-recorded beside the
        # headline: advection-diffusion 1024x1024x512 (fp32 and bf16 storage)
        # and the 256-grid batch against one grid per launch
        for name, st in (("advdiff_1024x1024x512_f32", wfa.F32), ("advdiff_1024x1024x512_bf16", wfa.BF16)):
            sub = grid_bench(args, workload("advdiff", 0), st, 1, 0, None, local, e2e=False,
                             accuracy=not args.no_accuracy)
            extras[name] = {k: sub[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "config",
                                                "roofline", "accuracy", "gpu_launches", "clocks")}
        extras["batch_256_grids"] = batch_bench(args, emit=False)
    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": r["config"], "roofline": r["roofline"], "linf_rel_err": r["accuracy"] and
                r["accuracy"]["linf_rel_err"], "accuracy": r["accuracy"], "cpu_baseline": cpu, "e2e": r["e2e"],
                "serving": serving, "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
        if extras:
            line["other_configs"] = extras
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def split_bench(args, rank, world, dist, local):
    """One grid split into slabs along z (Sec. 1 Fig. 1b domain
    decomposition): with N ranks each GPU holds one slab and the boundary
    planes move by NCCL send / receive before every step (strong scaling: the
    grid stays the same); on one GPU, --slabs slabs step through
    wfa_slabs_step (plane copies between slabs on the device)."""
    import numpy as np
    import torch

    import paper_2209_13768_gb300 as wfa
    from paper_2209_13768_gb300 import slabs
    p = workload(args.workload, args.solve_steps, args.shape)
    storage = wfa.BF16 if args.workload == "advdiff_bf16" else wfa.F32
    cells = p.shape[0] * p.shape[1] * p.shape[2]
    kvar = not np.isscalar(p.k)
    stream = torch.cuda.current_stream()
    if world > 1:
        s = slabs.DistSlab(dist, p.shape, rank, world, h=p.h, storage=storage, bc=p.bc)
        z0, z1 = s.z0, s.z1
        s.set_field(np.ascontiguousarray(p.T0[z0:z1]))
        s.set_coeffs(np.ascontiguousarray(p.k[z0:z1]) if kvar else p.k, p.u)
        nslabs = world
        interfaces = world if s.wrap else world - 1
    else:
        nslabs = args.slabs or 2
        # one stream per slab (their kernels overlap), timed on the first one:
        # wfa_slabs_step makes every slab's step wait for its neighbours' planes
        streams = [stream] + [torch.cuda.Stream() for _ in range(nslabs - 1)]
        s = slabs.SlabGrid(p.shape, nslabs, h=p.h, storage=storage, bc=p.bc,
                           streams=[st.cuda_stream or None for st in streams])
        s.set_field(p.T0)
        s.set_coeffs(p.k, p.u)
        interfaces = nslabs if p.bc[4][0] == "periodic" else nslabs - 1
    dt = p.dt if p.dt else 0.9 * s.stability_dt()
    s.set_dt(dt)
    for _ in range(args.warmup):
        s.step(p.steps)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    others = streams[1:] if world == 1 else []
    for i in range(args.steps):
        ev[i][0].record(stream)
        s.step(p.steps)
        for st in others:   # the other slabs' last steps end inside the timed step
            stream.wait_stream(st)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_s = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, dist, "cuda")
    value = cells * p.steps * args.steps / total_s / 1e9     # the whole grid, once (strong scaling)
    esize = 2 if storage == wfa.BF16 else 4
    plane = (p.shape[0] + 16 + 31) // 32 * 32 * (p.shape[1] + 16) * esize
    s.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "bf16" if storage == wfa.BF16 else "f32",
            "data": "synthetic",
            "config": {"workload": p.name, "cells": cells, "time_steps_per_step": p.steps, "dt": dt,
                       "decomposition": f"{nslabs} z slabs" + (" (one per GPU)" if world > 1 else " on one GPU"),
                       "exchange": ("NCCL send/recv of whole padded planes before every time step" if world > 1
                                    else "device copies of whole padded planes before every time step (wfa_slabs_step)"),
                       "exchange_bytes_per_time_step": 2 * interfaces * plane,
                       "parallelism": f"z slabs x{nslabs}"},
            "roofline": None, "gpu_launches": None, "clocks": clocks}), flush=True)


KERNEL_NAMES = {3: "sweep_col", 4: "sweep_col2 (two steps per pass)", 5: "sweep_col (boundaries in place)",
                6: "sweep_col (8 cells a thread; 16 for bf16 with uniform k)", 7: "sweep_t2 (two steps per pass, TMA-staged planes)",
                -1: "sweep_simple"}


def accuracy_boxes(p, edge=16):
    """Target boxes for the oracle comparison: the corners where the most
    faces meet, the middle of a face of every axis, and the grid's centre
    (where the advection-diffusion blob has its maximum)."""
    nx, ny, nz = p.shape
    e = [min(edge, n) for n in p.shape]
    mid = lambda n, w: (n - w) // 2
    corners = [(0, 0, 0), (nx - e[0], ny - e[1], nz - e[2]), (0, ny - e[1], nz - e[2]), (nx - e[0], 0, 0)]
    faces = [(0, mid(ny, e[1]), mid(nz, e[2])), (mid(nx, e[0]), 0, mid(nz, e[2])),
             (mid(nx, e[0]), mid(ny, e[1]), nz - e[2])]
    centre = [(mid(nx, e[0]), mid(ny, e[1]), mid(nz, e[2]))]
    return [(lo, (lo[0] + e[0], lo[1] + e[1], lo[2] + e[2])) for lo in corners + faces + centre]


def accuracy_sample(g, p, dt, storage, n):
    """L-inf error of the GPU field after an n-step prefix of the workload,
    relative to max |T| of the FP64 oracle, on sampled boxes (outside every
    timed region). The oracle steps each box widened by n cells (the
    stencil's domain of dependence, oracle/lightcone.py), so its values there
    are the whole-grid oracle's."""
    import numpy as np

    from oracle import lightcone
    kvar = not np.isscalar(p.k)
    t0 = time.perf_counter()
    g.set_field(p.T0)
    g.set_dt(dt)
    g.step(n)
    T = g.read_field()
    err, scale, cells = 0.0, 0.0, 0
    k = np.asarray(p.k) if kvar else float(p.k)
    for lo, hi in accuracy_boxes(p):
        ref = lightcone.run_box(p.T0, n, shape=p.shape, lo=lo, hi=hi, h=p.h, k=k, u=p.u, bc=p.bc, dt=dt)
        got = T[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].astype(np.float64)
        err = max(err, float(np.abs(got - ref).max()))
        scale = max(scale, float(np.abs(ref).max()))
        cells += ref.size
    rel = err / scale if scale > 0 else err
    bf16 = storage == 1
    bound = (n + 1) * 2.0 ** -9 if bf16 else 1e-5
    return {"linf_rel_err": rel, "bound": bound, "within_bound": rel <= bound, "steps": n,
            "reference": "FP64 oracle (oracle.run on each box widened by n cells)",
            "sample": f"{cells} cells in {len(accuracy_boxes(p))} boxes of up to 16^3 (corners, face middles, "
                      f"centre) after the first {n} time steps of the workload",
            "bound_reason": "(n+1) 2^-9 relative: bf16 storage rounds once at set-up and once a step, "
                            "the update is non-expansive" if bf16 else
                            "1e-5 after 100 steps (fp32 arithmetic, the update is non-expansive)",
            "seconds": time.perf_counter() - t0}


def grid_bench(args, p, storage, world, rank, dist, local, e2e=True, accuracy=True):
    """Time one single-grid workload (a benchmark step = p.steps time steps)
    and return its numbers: rate, roofline of the main sweep kernel, e2e
    through the C ABI from pinned host buffers, accuracy against the oracle."""
    import numpy as np
    import torch

    import paper_2209_13768_gb300 as wfa
    kvar = not np.isscalar(p.k)
    cells = p.shape[0] * p.shape[1] * p.shape[2]
    stream = torch.cuda.Stream()
    g = wfa.Grid(p.shape, h=p.h, storage=storage, stream=stream.cuda_stream)
    g.set_bcs(p.bc)
    g.set_coeffs(p.k, p.u)
    g.set_field(p.T0)
    dt = p.dt if p.dt else 0.9 * g.stability_dt()
    g.set_dt(dt)
    g.set_tuning(args.depth, args.variant)
    g.set_zchunk(args.zchunk)
    if not (args.depth or args.variant or args.zchunk):
        g.autotune()   # time the compiled configurations on this grid, keep the fastest
    depth, variant, zchunk = g.tuning()
    passes_per_step = math.ceil(p.steps / depth)

    for _ in range(args.warmup):
        g.step(p.steps)
    g.sync()

    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # the dominant kernel's own launches are bracketed by events inside the
    # library, on the grid's stream: every 16th pass, at most about 4000 samples
    g.set_kernel_timing(max(16, math.ceil(args.steps * passes_per_step / 4000)))
    launches0 = g.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for i in range(args.steps):
        ev[i][0].record(stream)
        g.step(p.steps)
        ev[i][1].record(stream)
    g.sync()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    kernel_ms, kernel_launches = g.kernel_time()
    gpu_launches = g.launch_count() - launches0   # every kernel of the timed steps
    g.set_kernel_timing(0)
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    total_s = max_over_ranks(total_s, dist, "cuda")
    value = job_rate(world, cells * p.steps * args.steps, total_s)

    # roofline of the dominant kernel (the main sweep): algorithmic bytes per
    # launch (read T, read k, write T once per pass) over its mean duration,
    # from the event pairs the library recorded around its sampled launches.
    # When the main kernel is the pass's only kernel, the pass mean (no event
    # records inside) bounds its duration from above and is the tighter figure.
    pass_s = total_s / (args.steps * passes_per_step)
    launch_s = kernel_ms / 1e3 / kernel_launches if kernel_launches else pass_s
    launches_per_pass = gpu_launches / max(1, args.steps * passes_per_step)
    event_s = launch_s
    if launches_per_pass <= 1.0 + 1e-9:
        launch_s = min(launch_s, pass_s)
    bpc = bytes_per_cell(storage == wfa.BF16, kvar)
    achieved = bpc * cells / launch_s / 1e9
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    traffic = None
    try:
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
        key = (f"{'bf16' if storage else 'f32'}:{'k' if kvar else 'u'}:{'adv' if any(p.u) else 'noadv'}"
               f":v{variant}:d{depth}:{p.shape[0]}x{p.shape[1]}x{p.shape[2]}")
        ent = tr.get(key)
        if ent and ent.get("kernel_hash") == kernel_hash() and ent.get("zchunk", 0) == zchunk:
            traffic = ent["bytes_per_launch"]
    except (OSError, ValueError):
        pass
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "bytes_per_cell_per_launch": bpc, "steps_per_launch": depth,
                "kernel_ms_mean": launch_s * 1e3, "kernel_ms_mean_event_pairs": event_s * 1e3,
                "kernel_launches_timed": kernel_launches, "launches_per_pass": launches_per_pass,
                # DRAM bytes per launch from ncu over this run's mean launch time
                "ncu_dram_GBps": traffic / launch_s / 1e9 if traffic else None,
                "ncu_dram_frac": traffic / launch_s / 1e9 / peak if traffic else None,
                "traffic_over_algorithmic": traffic / (bpc * cells) if traffic else None,
                "pass_ms_mean": pass_s * 1e3, "pass_GBps": bpc * cells / pass_s / 1e9,
                "effective_GBps_paper_Teff": bpc * depth * cells / pass_s / 1e9,
                "frac_of_nominal_8TBps": achieved / 8000.0}

    # end to end through the C ABI from pinned host buffers
    e2e_line = None
    if e2e:
        T0h = torch.from_numpy(np.ascontiguousarray(p.T0)).pin_memory()
        kh = torch.from_numpy(np.ascontiguousarray(p.k)).pin_memory() if kvar else None
        outh = torch.empty(tuple(p.T0.shape), dtype=torch.float32).pin_memory()
        nrep = max(1, min(args.steps, 3))
        e2e_t = []
        parts = {"set_field": [], "set_coeffs": [], "set_dt": [], "step": [], "read_field": []}
        for i in range(nrep + 1):
            torch.cuda.synchronize()
            t = [time.perf_counter()]
            g.set_field(T0h)                          # returns once the host buffer was read
            t.append(time.perf_counter())
            g.set_coeffs(kh if kvar else p.k, p.u)    # validates k on the device: synchronous
            t.append(time.perf_counter())
            g.set_dt(dt)                              # checks dt against the fp64 limit: synchronous
            t.append(time.perf_counter())
            g.step(p.steps)
            g.sync()                                  # only to time the pieces; read_field waits anyway
            t.append(time.perf_counter())
            g.read_field(outh)
            t.append(time.perf_counter())
            if i:   # first one is a warm-up
                e2e_t.append(t[-1] - t[0])
                for k, (a, b) in zip(parts, zip(t, t[1:])):
                    parts[k].append(1e3 * (b - a))
        e2e_s = sum(e2e_t) / len(e2e_t)
        e2e_s = max_over_ranks(e2e_s, dist, "cuda")
        e2e_line = {"value": job_rate(world, cells * p.steps, e2e_s), "unit": "GLUPS",
                    "h2d_bytes_per_step": cells * 4 * (2 if kvar else 1), "d2h_bytes_per_step": cells * 4,
                    "ms_per_step": 1e3 * e2e_s,
                    "ms_by_call": {k: sum(v) / len(v) for k, v in parts.items()}}
    acc = None
    if accuracy and rank == 0:
        acc = accuracy_sample(g, p, dt, storage, min(100, p.steps))
    g.close()
    config = {"workload": p.name, "cells": cells, "time_steps_per_step": p.steps, "depth": depth,
              "kernel": KERNEL_NAMES.get(variant, f"sweep_tb variant {variant}"), "variant": variant,
              "zchunk": zchunk or "automatic", "dt": dt, "storage": "bf16" if storage else "f32",
              "conductivity": "per-cell lognormal(0,0.5)" if kvar else f"uniform {p.k}",
              "l2": "inputs larger than L2 (%.0f MiB field)" % (cells * (2 if storage else 4) / 2**20),
              "parallelism": f"replicas x{world}"}
    return {"value": value, "unit": "GLUPS", "ms_per_step": 1e3 * total_s / args.steps, "steps": args.steps,
            "warmup": args.warmup, "config": config, "roofline": roofline, "accuracy": acc, "e2e": e2e_line,
            "gpu_launches": gpu_launches, "clocks": clocks}


if __name__ == "__main__":
    main()
