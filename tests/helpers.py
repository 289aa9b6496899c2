"""Shared test helpers: run a Problem on the GPU library and on the oracle."""
import numpy as np

import oracle
import paper_2209_13768_gb300 as wfa


def rel_linf(a, ref):
    """max |a - ref| / max |ref| (the error measure of every parity check)."""
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    return float(np.abs(np.asarray(a, dtype=np.float64) - ref).max() / (scale if scale > 0 else 1.0))


def oracle_dt(p):
    if p.dt:
        return p.dt
    return p.dt_factor * oracle.dt_max(shape=p.shape, h=p.h, k=_k64(p.k), u=p.u, bc=p.bc)


def _k64(k):
    return k if np.isscalar(k) else np.asarray(k, dtype=np.float64)


def run_oracle(p, steps=None, dt=None, round_to=None, T0=None):
    steps = p.steps if steps is None else steps
    dt = oracle_dt(p) if dt is None else dt
    return oracle.run(p.T0 if T0 is None else T0, steps, shape=p.shape, h=p.h, k=_k64(p.k), u=p.u,
                      bc=p.bc, dt=dt, round_to=round_to)


def make_grid(p, storage=wfa.F32, depth=0, variant=0, dt=None, zchunk=0):
    g = wfa.Grid(p.shape, h=p.h, storage=storage)
    g.set_bcs(p.bc)
    g.set_coeffs(p.k, p.u)
    g.set_field(p.T0)
    if dt is None:
        dt = p.dt if p.dt else p.dt_factor * g.stability_dt()
    g.set_dt(dt)
    g.set_tuning(depth, variant)
    g.set_zchunk(zchunk)
    return g


def run_gpu(p, steps=None, storage=wfa.F32, depth=0, variant=0, dt=None, zchunk=0):
    steps = p.steps if steps is None else steps
    with make_grid(p, storage, depth, variant, dt, zchunk) as g:
        g.step(steps)
        return g.read_field()
