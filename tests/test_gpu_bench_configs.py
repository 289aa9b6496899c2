"""Parity at the benchmark configurations themselves, against the FP64 oracle.

* Heat with lognormal k at the full 512^3: every cell after a 100-step prefix
  of the 1000-step run (the oracle takes tens of seconds for the prefix; the
  full 1000 steps would take minutes), in the launch configuration bench.py
  times (autotuned).
* Advection-diffusion at the full 1024 x 1024 x 512, fp32 and bf16 storage:
  a 100-step prefix on boxes at the corners, face middles and centre, the
  oracle stepping each box widened by 100 cells (domain of dependence,
  oracle/lightcone.py).
* The 256-grid batch exactly as benchmarked (edges log-uniform in [16, 128],
  50 to 500 steps each): every grid bitwise equal to the grid stepped alone,
  and every grid against the oracle.
* The continuous-batching server: every result against the oracle directly.

Tolerances as everywhere: fp32 <= 1e-5 of max |T| (relative L-inf); bf16
storage <= (n + 1) 2^-9 against the plain fp64 oracle and within a few bf16
ulps of the oracle that rounds to bf16 after every step."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
import paper_2209_13768_gb300 as wfa
from oracle import lightcone
from paper_2209_13768_gb300 import workloads as W
from helpers import rel_linf

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
CORES = os.cpu_count() or 1


def _boxes(shape, edge=16):
    nx, ny, nz = shape
    e = [min(edge, n) for n in shape]
    mid = lambda n, w: (n - w) // 2
    los = [(0, 0, 0), (nx - e[0], ny - e[1], nz - e[2]), (0, ny - e[1], nz - e[2]), (nx - e[0], 0, 0),
           (0, mid(ny, e[1]), mid(nz, e[2])), (mid(nx, e[0]), 0, mid(nz, e[2])),
           (mid(nx, e[0]), mid(ny, e[1]), nz - e[2]), (mid(nx, e[0]), mid(ny, e[1]), mid(nz, e[2]))]
    return [(lo, (lo[0] + e[0], lo[1] + e[1], lo[2] + e[2])) for lo in los]


def test_lognormal_512_every_cell_after_100_steps():
    p = W.heat_lognormal()                   # 512^3, per-cell k, x Dirichlet 1 / 0, y / z zero flux
    n = 100
    with wfa.Grid(p.shape) as g:
        g.set_bcs(p.bc)
        g.set_coeffs(p.k, p.u)
        g.set_field(p.T0)
        dt = 0.9 * g.stability_dt()
        g.set_dt(dt)
        choice = g.autotune()                 # the configuration bench.py times
        g.step(n)
        T = g.read_field()
    ref = oracle.run(p.T0, n, shape=p.shape, k=np.asarray(p.k, dtype=np.float64), bc=p.bc, dt=dt)
    err = rel_linf(T, ref)
    assert err <= F32_TOL, (err, choice)


@pytest.mark.parametrize("storage", [wfa.F32, wfa.BF16])
def test_advection_diffusion_1024_boxes_after_100_steps(storage):
    p = W.advection_diffusion()               # 1024 x 1024 x 512, uniform k, periodic x
    n = 100
    with wfa.Grid(p.shape, h=p.h, storage=storage) as g:
        g.set_bcs(p.bc)
        g.set_coeffs(p.k, p.u)
        g.set_field(p.T0)
        g.set_dt(p.dt)
        choice = g.autotune()
        g.step(n)
        T = g.read_field()
    err, scale, ulps = 0.0, 0.0, 0.0
    boxes = _boxes(p.shape)
    for lo, hi in boxes:
        got = T[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].astype(np.float64)
        ref = lightcone.run_box(p.T0, n, shape=p.shape, lo=lo, hi=hi, h=p.h, k=p.k, u=p.u, bc=p.bc, dt=p.dt)
        err = max(err, float(np.abs(got - ref).max()))
        scale = max(scale, float(np.abs(ref).max()))
        if storage == wfa.BF16 and (lo, hi) == boxes[-1]:   # the centre box, around the blob
            refb = lightcone.run_box(p.T0, n, shape=p.shape, lo=lo, hi=hi, h=p.h, k=p.k, u=p.u, bc=p.bc, dt=p.dt,
                                     round_to="bf16")
            ulp = 2.0 ** -7 * np.maximum(np.abs(refb), 2.0 ** -126)
            ulps = max(ulps, float(np.max(np.abs(got - refb) / ulp)))
    bound = F32_TOL if storage == wfa.F32 else (n + 1) * 2.0 ** -9
    assert err / scale <= bound, (err / scale, choice)
    if storage == wfa.BF16:
        assert ulps <= 4.0, (ulps, choice)


def _oracle_grid(p, n, dt):
    k = p.k if np.isscalar(p.k) else np.asarray(p.k, dtype=np.float64)
    return oracle.run(p.T0, n, shape=p.shape, h=p.h, k=k, u=p.u, bc=p.bc, dt=dt, threads=1)


def test_batch_256_grids_as_benchmarked():
    probs = W.batch_grids()                   # 256 grids, edges 16..128, steps 50..500
    grids = []
    try:
        for p in probs:
            g = wfa.Grid(p.shape)
            g.set_bcs(p.bc)
            g.set_coeffs(p.k, p.u)
            g.set_field(p.T0)
            g.set_dt(0.9 * g.stability_dt())
            grids.append(g)
        dts = [0.9 * g.stability_dt() for g in grids]
        wfa.batch_run(grids, [p.steps for p in probs])
        fields = [g.read_field() for g in grids]
    finally:
        for g in grids:
            g.close()
    for p, dt, T in zip(probs, dts, fields):    # bitwise: each grid stepped alone
        with wfa.Grid(p.shape) as g:
            g.set_bcs(p.bc)
            g.set_coeffs(p.k, p.u)
            g.set_field(p.T0)
            g.set_dt(dt)
            g.step(p.steps)
            np.testing.assert_array_equal(T, g.read_field(), err_msg=f"{p.name} {p.shape} {p.steps} steps")
    with cf.ThreadPoolExecutor(CORES) as ex:   # the oracle, one grid per host core
        refs = list(ex.map(lambda a: _oracle_grid(*a), [(p, p.steps, dt) for p, dt in zip(probs, dts)]))
    errs = [rel_linf(T, ref) for T, ref in zip(fields, refs)]
    assert max(errs) <= F32_TOL, (max(errs), int(np.argmax(errs)))


def test_server_results_match_oracle():
    """Requests from the serving stream (both physics, fp32 and bf16), edges
    and step counts cut down so that the oracle stays quick; each result on
    the host against the oracle run on the same request."""
    arrivals = W.request_stream(rate=1000.0, count=16, lo=20, hi=56, steps=(20, 120), seed=15)
    with wfa.Server(budget_bytes=4 << 30, quantum=16) as srv:
        tickets = [(srv.submit(a.problem.shape, a.problem.T0, a.problem.steps, h=a.problem.h, storage=a.storage,
                               k=a.problem.k, u=a.problem.u, bc=a.problem.bc, dt=a.problem.dt), a) for a in arrivals]
        outs = [(srv.wait(t, timeout=120), a) for t, a in tickets]
    kinds = set()
    for out, a in outs:
        p = a.problem
        kk = p.k if np.isscalar(p.k) else np.asarray(p.k, dtype=np.float64)
        dt = p.dt if p.dt else 0.9 * oracle.dt_max(shape=p.shape, h=p.h, k=kk, u=p.u, bc=p.bc)
        ref = oracle.run(p.T0, p.steps, shape=p.shape, h=p.h, k=kk, u=p.u, bc=p.bc, dt=dt)
        err = rel_linf(out, ref)
        if a.storage == wfa.F32:
            assert err <= F32_TOL, (p.name, p.shape, p.steps, err)
        else:
            assert err <= (p.steps + 1) * 2.0 ** -9, (p.name, p.shape, p.steps, err)
            refb = oracle.run(oracle.round_to(p.T0, "bf16"), p.steps, shape=p.shape, h=p.h, k=kk, u=p.u, bc=p.bc,
                              dt=dt, round_to="bf16")
            ulp = 2.0 ** -7 * np.maximum(np.abs(refb), 2.0 ** -126)
            assert np.max(np.abs(out - refb) / ulp) <= 4.0, (p.name, p.shape, p.steps)
        kinds.add((p.name, a.storage))
    assert len(kinds) == 4   # heat and advection-diffusion, fp32 and bf16 all present
