"""Parity at the benchmark sizes, in the launch configuration bench.py times.

The oracle cannot run 512^3 or 1024^2 x 512 grids for hundreds of steps, but
after n steps a cell depends only on the cells within n of it (the stencil
reaches one neighbour per step). So for sampled cells the oracle runs on the
(2n+1)^3 box around the cell, cut out of the full inputs: real boundary
faces keep their condition, the cut faces get any condition (zero flux here)
because their influence cannot reach the centre within n steps. The GPU runs
the whole grid; the two are compared cell by cell at the samples."""
import numpy as np
import pytest

import oracle
import paper_2209_13768_gb300 as wfa
from paper_2209_13768_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ZF = W.ZF


def _samples(shape, count, rng):
    """Random cells plus every corner and cells on each face and edge."""
    nx, ny, nz = shape
    pts = [tuple(int(v) for v in (rng.integers(0, nx), rng.integers(0, ny), rng.integers(0, nz)))
           for _ in range(count)]
    ends = lambda n: (0, 1, n // 2, n - 2, n - 1)
    pts += [(x, y, z) for x in ends(nx) for y in ends(ny) for z in ends(nz)]
    return sorted(set(pts))


def _cone_box(p, cell, n, k_full, T_full):
    """Inputs and faces of the box of radius n around cell, and the cell's
    position in it."""
    idx, faces, centre, shape = [], [], [], []
    for a in range(3):
        N, c = p.shape[a], cell[a]
        lo_kind, hi_kind = p.bc[2 * a], p.bc[2 * a + 1]
        periodic = lo_kind[0] == W.P
        if periodic and 2 * n + 1 >= N:
            ix = np.arange(N)
            faces += [lo_kind, hi_kind]
            centre.append(c)
        elif periodic:
            ix = np.arange(c - n, c + n + 1) % N
            faces += [(ZF, 0.0), (ZF, 0.0)]
            centre.append(n)
        else:
            lo, hi = max(0, c - n), min(N - 1, c + n)
            ix = np.arange(lo, hi + 1)
            faces += [lo_kind if lo == 0 else (ZF, 0.0), hi_kind if hi == N - 1 else (ZF, 0.0)]
            centre.append(c - lo)
        idx.append(ix)
        shape.append(len(ix))
    sel = np.ix_(idx[2], idx[1], idx[0])
    k = k_full if np.isscalar(k_full) else np.asarray(k_full[sel], np.float64)
    return tuple(shape), T_full[sel].astype(np.float64), k, faces, centre


def _oracle_at(p, cells, n, dt, T0, round_to=None):
    out = []
    for cell in cells:
        shape, T, k, faces, (cx, cy, cz) = _cone_box(p, cell, n, p.k, T0)
        if round_to:   # the initial rounding is per cell: round the box only
            T = oracle.round_to(T, round_to).astype(np.float64)
        R = oracle.run(T, n, shape=shape, h=p.h, k=k, u=p.u, bc=faces, dt=dt, round_to=round_to)
        out.append(R[cz, cy, cx])
    return np.array(out)


def _gpu_field(p, n, storage, depth, variant, dt):
    with wfa.Grid(p.shape, h=p.h, storage=storage) as g:
        g.set_bcs(p.bc)
        g.set_coeffs(p.k, p.u)
        g.set_field(p.T0)
        g.set_dt(dt)
        if depth == 0 and variant == 0:
            depth, variant = g.autotune()     # what bench.py does
        else:
            g.set_tuning(depth, variant)
        g.step(n)
        return g.read_field(), (depth, variant)


def test_lognormal_512_sampled_parity():
    p = W.heat_lognormal()                    # 512^3, per-cell k, x Dirichlet, y / z zero flux
    n = 6
    with wfa.Grid(p.shape) as g:
        g.set_bcs(p.bc)
        g.set_coeffs(p.k, p.u)
        dt = 0.9 * g.stability_dt()
    T, choice = _gpu_field(p, n, wfa.F32, 0, 0, dt)
    rng = np.random.default_rng(31)
    cells = _samples(p.shape, 1500, rng)
    ref = _oracle_at(p, cells, n, dt, p.T0)
    got = np.array([T[z, y, x] for x, y, z in cells])
    scale = max(np.abs(ref).max(), 1.0)
    assert np.max(np.abs(got - ref)) / scale <= 1e-5, choice
    # the other kernels give the same field bit for bit at this size
    for depth, variant in [(1, 3), (2, 1), (4, 2)]:
        if (depth, variant) != choice:
            T2, _ = _gpu_field(p, n, wfa.F32, depth, variant, dt)
            np.testing.assert_array_equal(T2, T, err_msg=f"depth {depth} variant {variant}")


@pytest.mark.parametrize("storage", [wfa.F32, wfa.BF16])
def test_advection_diffusion_1024_sampled_parity(storage):
    p = W.advection_diffusion()               # 1024 x 1024 x 512, uniform k, periodic x
    n = 5
    T, choice = _gpu_field(p, n, storage, 0, 0, p.dt)
    rng = np.random.default_rng(32)
    cells = _samples(p.shape, 600, rng)
    # cells near the blob, where the field is not ~0
    nx, ny, nz = p.shape
    cells += [(nx // 2 + int(dx), ny // 2 + int(dy), nz // 2 + int(dz)) for dx, dy, dz in rng.integers(-40, 40, (300, 3))]
    got = np.array([T[z, y, x] for x, y, z in cells])
    if storage == wfa.F32:
        ref = _oracle_at(p, cells, n, p.dt, p.T0)
        assert np.max(np.abs(got - ref)) / np.abs(ref).max() <= 1e-5, choice
    else:
        # the oracle with the same per-step bf16 rounding: a few bf16 ulps apart
        ref = _oracle_at(p, cells, n, p.dt, p.T0, round_to="bf16")
        ulp = 2.0 ** -7 * np.maximum(np.abs(ref), 2.0 ** -126)
        assert np.max(np.abs(got - ref) / ulp) <= 4.0, choice
