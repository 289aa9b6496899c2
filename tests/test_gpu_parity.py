"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances. FP32 fields: L-infinity error relative to max |T| <= 1e-5 after
100 steps (the update is a convex combination for dt <= dt_max, so per-step
fp32 rounding, ~6e-8 relative, adds up at most linearly: 100 steps stay well
below 1e-5). BF16 storage: <= (n + 1) * 2^-9 relative (initial rounding plus
one nearest-even rounding per step, propagated without growth by the same
non-expansive update), and against the oracle run with the same per-step
bf16 rounding, within a few bf16 ulps where fp32 vs fp64 arithmetic tips a
rounding. Across kernels (tile shapes, temporal depths, the one-column
kernel) the per-cell expression is fixed, so fields must be bit-identical.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import paper_2209_13768_gb300 as wfa
from paper_2209_13768_gb300 import workloads as W
from helpers import make_grid, oracle_dt, rel_linf, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

D, ZF, P, DC = W.D, W.ZF, W.P, W.DC
F32_TOL = 1e-5
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bf16_bound(steps):
    return (steps + 1) * 2.0**-9


# ------------------------------------------------------------ heat 64^3 --
@pytest.mark.parametrize("held", [False, True])
def test_heat64_matches_oracle(held):
    p = W.heat_64(held_cells=held)
    ref = run_oracle(p)
    assert abs(oracle_dt(p) - (0.9 / 6 if held else 0.1)) < 1e-15
    outs = {}
    for variant, depth in [(-1, 1), (1, 1), (1, 2), (1, 4), (2, 3), (1, 8), (2, 8), (3, 1), (0, 0)]:
        T = run_gpu(p, depth=depth, variant=variant)
        err = rel_linf(T, ref)
        assert err <= F32_TOL, (variant, depth, err)
        outs[(variant, depth)] = T
    base = outs[(-1, 1)]
    for key, T in outs.items():
        np.testing.assert_array_equal(T, base, err_msg=str(key))


def test_heat64_dt_limit_on_gpu():
    p = W.heat_64()
    with make_grid(p) as g:
        assert abs(g.stability_dt() - 1.0 / 9.0) < 1e-15
    p = W.heat_64(held_cells=True)
    with make_grid(p) as g:
        assert abs(g.stability_dt() - 1.0 / 6.0) < 1e-15


# ----------------------------------------------------- every boundary mix --
MIXES = [
    [(D, 0.3), (D, -0.7), (D, 1.0), (D, 0.0), (D, 0.5), (D, 2.0)],
    [(ZF, 0)] * 6,
    [(P, 0)] * 6,
    [(DC, 0.25), (DC, 0.75), (DC, -0.5), (DC, 1.0), (DC, 0.1), (DC, 0.2)],
    [(D, 1.0), (ZF, 0), (P, 0), (P, 0), (DC, 0.5), (D, 0.0)],
    [(DC, 1.0), (D, 0.0), (ZF, 0), (DC, 0.3), (P, 0), (P, 0)],
    [(P, 0), (P, 0), (D, 0.2), (ZF, 0), (ZF, 0), (D, 0.8)],
]


def _mixed_problem(mix, shape=(37, 29, 23), kvar=True, adv=True, seed=0):
    rng = np.random.default_rng(1000 + seed)
    nx, ny, nz = shape
    k = np.exp(0.5 * rng.standard_normal((nz, ny, nx))).astype(np.float32) if kvar else 0.8
    u = tuple(rng.uniform(-0.4, 0.4, 3)) if adv else (0.0, 0.0, 0.0)
    h = tuple(rng.uniform(0.8, 1.25, 3))
    T0 = rng.uniform(0, 1, (nz, ny, nx)).astype(np.float32)
    return W.Problem(shape=shape, T0=T0, k=k, u=u, bc=MIXES[mix], h=h, steps=20)


@pytest.mark.parametrize("kvar,adv", [(True, True), (False, True), (True, False), (False, False)])
@pytest.mark.parametrize("mix", range(len(MIXES)))
def test_boundary_mixes_all_kernels(mix, kvar, adv):
    p = _mixed_problem(mix, kvar=kvar, adv=adv, seed=mix)
    ref = run_oracle(p)
    base = run_gpu(p, variant=-1)
    assert rel_linf(base, ref) <= F32_TOL
    for variant in (1, 2):
        for depth in range(1, 9):
            T = run_gpu(p, depth=depth, variant=variant)
            np.testing.assert_array_equal(T, base, err_msg=f"variant {variant} depth {depth}")
    np.testing.assert_array_equal(run_gpu(p, variant=3), base, err_msg="column kernel")
    # two-step column kernel (uniform k; per-cell k falls back to one step)
    np.testing.assert_array_equal(run_gpu(p, depth=2, variant=4), base, err_msg="two-step column kernel")
    np.testing.assert_array_equal(run_gpu(p, depth=2, variant=7), base, err_msg="two-step TMA kernel")
    np.testing.assert_array_equal(run_gpu(p, variant=5), base, err_msg="column kernel, boundaries in place")
    np.testing.assert_array_equal(run_gpu(p, variant=6), base, err_msg="column kernel, 8 cells a thread")
    np.testing.assert_array_equal(run_gpu(p, steps=p.steps - 1, depth=2, variant=4),
                                  run_gpu(p, steps=p.steps - 1, variant=-1), err_msg="two-step, odd count")
    np.testing.assert_array_equal(run_gpu(p, steps=p.steps - 1, depth=2, variant=7),
                                  run_gpu(p, steps=p.steps - 1, variant=-1), err_msg="two-step TMA, odd count")


@pytest.mark.parametrize("kvar,adv", [(True, True), (False, True), (True, False)])
@pytest.mark.parametrize("mix", range(len(MIXES)))
def test_column_kernel_z_chunks(mix, kvar, adv):
    """The column kernels march z chunks of any length, neighbouring chunks
    in opposite directions: the field is bitwise the same for every chunk
    length (one plane, odd lengths, a ragged last chunk, one chunk)."""
    p = _mixed_problem(mix, kvar=kvar, adv=adv, seed=50 + mix)
    base = run_gpu(p, variant=-1)
    for zc in (1, 2, 3, 5, 8, 12, 22, 23, 64):
        np.testing.assert_array_equal(run_gpu(p, variant=3, zchunk=zc), base, err_msg=f"variant 3, zchunk {zc}")
        np.testing.assert_array_equal(run_gpu(p, variant=5, zchunk=zc), base, err_msg=f"variant 5, zchunk {zc}")
        np.testing.assert_array_equal(run_gpu(p, depth=2, variant=7, zchunk=zc), base, err_msg=f"variant 7, zchunk {zc}")
        np.testing.assert_array_equal(run_gpu(p, variant=6, zchunk=zc), base, err_msg=f"variant 6, zchunk {zc}")
    for storage in (wfa.BF16,):
        ref = run_gpu(p, storage=storage, variant=-1)
        for zc in (3, 8, 12):
            np.testing.assert_array_equal(run_gpu(p, storage=storage, variant=3, zchunk=zc), ref,
                                          err_msg=f"bf16 zchunk {zc}")


@pytest.mark.parametrize("kvar", [True, False])
@pytest.mark.parametrize("mix", [2, 4, 5, 6])
def test_kernel_switches_between_thin_and_full_periodic_copies(mix, kvar):
    """The one-step column passes write one layer of periodic copies; a tiled
    or two-step pass after them needs every layer (and the corners): the
    switch completes the copies first, so any sequence of kernels gives the
    field of one kernel throughout."""
    p = _mixed_problem(mix, kvar=kvar, seed=70 + mix)
    plan = [(1, 3, 3), (2, 7, 4), (2, 1, 2), (1, 6, 2), (2, 7, 3), (3, 2, 3), (1, 5, 1), (2, 4, 2), (1, 3, 1),
            (2, 7, 2)]   # (depth, variant, steps)
    ref = run_gpu(p, steps=sum(n for _, _, n in plan), variant=-1)
    with make_grid(p) as g:
        for depth, variant, steps in plan:
            g.set_tuning(depth, variant)
            g.step(steps)
        np.testing.assert_array_equal(g.read_field(), ref)


@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 2, 5), (5, 7, 3), (64, 3, 9), (131, 67, 4), (70, 35, 40)])
def test_small_and_ragged_shapes(shape):
    for mix in (0, 2, 4):
        if any(k == DC for k, _ in MIXES[mix]) and min(shape) < 3:
            continue
        p = _mixed_problem(mix, shape=shape, seed=7)
        p.steps = 9
        ref = run_oracle(p)
        base = run_gpu(p, variant=-1)
        assert rel_linf(base, ref) <= F32_TOL
        for depth in (1, 3, 8):
            np.testing.assert_array_equal(run_gpu(p, depth=depth, variant=1), base)
        np.testing.assert_array_equal(run_gpu(p, variant=3), base)
        np.testing.assert_array_equal(run_gpu(p, variant=5), base)
        np.testing.assert_array_equal(run_gpu(p, variant=6), base)
        pu = _mixed_problem(mix, shape=shape, kvar=False, seed=7)
        pu.steps = 9
        np.testing.assert_array_equal(run_gpu(pu, depth=2, variant=4), run_gpu(pu, variant=-1), err_msg=str(shape))
        np.testing.assert_array_equal(run_gpu(pu, depth=2, variant=7), run_gpu(pu, variant=-1), err_msg=str(shape))



GHOST_MIX = [(D, 0.5), (D, -0.75), (ZF, 0), (D, 1.0), (D, 0.0), (ZF, 0)]   # values exact in bf16


@pytest.mark.parametrize("storage", [wfa.F32, wfa.BF16])
def test_ghost_layer_boundaries(storage):
    # per-cell k without advection and Dirichlet values a bf16 halo holds
    # exactly: the column kernel reads the boundary conditions from ghost
    # layers (k = inf beside a Dirichlet face, k = 0 beside a zero-flux one)
    for shape in [(37, 29, 23), (6, 5, 9), (64, 16, 16), (2, 3, 2)]:
        p = _mixed_problem(0, shape=shape, kvar=True, adv=False, seed=11)
        p.bc = GHOST_MIX
        base = run_gpu(p, storage=storage, variant=-1)
        np.testing.assert_array_equal(run_gpu(p, storage=storage, variant=3), base, err_msg=str(shape))
        if storage == wfa.F32:
            assert rel_linf(base, run_oracle(p)) <= F32_TOL
    # boundary conditions changed between steps (odd counts leave the field in
    # either buffer): both buffers' ghost layers follow every change
    p = _mixed_problem(0, kvar=True, adv=False, seed=12)
    p.bc = GHOST_MIX
    changes = [[], [(0, ZF, 0.0)], [(2, D, 0.25)], [(0, P, 0.0), (1, P, 0.0)], [(5, D, -1.0)], [(3, DC, 0.5)],
               [(3, D, 0.5), (0, D, 2.0), (1, ZF, 0.0)]]
    grids = [make_grid(p, storage=storage, variant=v) for v in (3, -1)]
    try:
        for change in changes:
            for g in grids:
                for face, kind, value in change:
                    g.set_bc(face, kind, value)
                if change:
                    g.set_dt(0.5 * g.stability_dt())
                g.step(3)
            np.testing.assert_array_equal(grids[0].read_field(), grids[1].read_field(), err_msg=f"after {change}")
    finally:
        for g in grids:
            g.close()


def test_zero_steps_and_step_accounting():
    p = _mixed_problem(4)
    with make_grid(p) as g:
        g.step(0)
        T = g.read_field()
        held = oracle.run(p.T0, 0, shape=p.shape, h=p.h, k=np.asarray(p.k, np.float64), u=p.u, bc=p.bc, dt=0.1)
        np.testing.assert_array_equal(T, held.astype(np.float32))
        g.step(5)
        g.step(6)
        assert g.steps_done() == 11
        np.testing.assert_array_equal(g.read_field(), run_gpu(p, steps=11))


# -------------------------------------------------------------- bf16 ------
@pytest.mark.parametrize("mix", [0, 2, 4])
def test_bf16_storage(mix):
    p = _mixed_problem(mix, seed=3)
    p.steps = 30
    ref = run_oracle(p)
    ref_rounded = run_oracle(p, round_to="bf16", T0=oracle.round_to(p.T0, "bf16"))
    base = run_gpu(p, storage=wfa.BF16, variant=-1)
    assert rel_linf(base, ref) <= bf16_bound(p.steps)
    # same per-step rounding as the oracle diagnostic: at most a few bf16 ulps apart
    ulp = 2.0**-7 * np.maximum(np.abs(ref_rounded), 2.0**-126)
    assert np.max(np.abs(base - ref_rounded) / ulp) <= 4.0
    for depth in (1, 2, 5, 8):
        for variant in (1, 2):
            np.testing.assert_array_equal(run_gpu(p, storage=wfa.BF16, depth=depth, variant=variant), base)
    np.testing.assert_array_equal(run_gpu(p, storage=wfa.BF16, variant=3), base)
    np.testing.assert_array_equal(run_gpu(p, storage=wfa.BF16, variant=5), base)
    pu = _mixed_problem(mix, kvar=False, seed=3)
    pu.steps = 30
    np.testing.assert_array_equal(run_gpu(pu, storage=wfa.BF16, depth=2, variant=7),
                                  run_gpu(pu, storage=wfa.BF16, variant=-1))
    np.testing.assert_array_equal(run_gpu(pu, storage=wfa.BF16, depth=2, variant=4),
                                  run_gpu(pu, storage=wfa.BF16, variant=-1))


# ------------------------------------------------------ reductions (fp64) --
def test_stability_dt_matches_oracle():
    for mix in range(len(MIXES)):
        p = _mixed_problem(mix, seed=11)
        ref = oracle.dt_max(shape=p.shape, h=p.h, k=np.asarray(p.k, np.float64), u=p.u, bc=p.bc)
        with make_grid(p) as g:
            got = g.stability_dt()
        assert abs(got - ref) <= 1e-13 * ref, (mix, got, ref)



@pytest.mark.parametrize("case", ["layered", "extreme", "zeros", "tiny_h", "uniform"])
def test_stability_dt_two_pass_cases(case):
    # per-cell k takes an fp32 pass, then fp64 on the near-maximal cells only;
    # ties, k values outside the fp32 pass's range, zero k and cell sizes that
    # send it to the one-pass fp64 reduction must all give the fp64 maximum
    rng = np.random.default_rng(21)
    shape = (23, 17, 12)
    nx, ny, nz = shape
    for mix in range(len(MIXES)):
        p = _mixed_problem(mix, shape=shape, seed=mix)
        if case == "layered":
            p.k = np.broadcast_to(rng.uniform(0.5, 2.0, nx).astype(np.float32), (nz, ny, nx)).copy()
        elif case == "extreme":
            k = np.asarray(p.k).copy()
            k[3, 4, 5], k[7, 2, 9], k[0, 0, 0] = 1e20, 1e-20, 3e16
            p.k = k
        elif case == "zeros":
            k = np.asarray(p.k).copy()
            k[rng.random(k.shape) < 0.3] = 0.0
            p.k = k
        elif case == "tiny_h":
            p.h = (1e-9, 2e-9, 1.5e-9)
        else:
            p.k = 0.7
        k = p.k if np.isscalar(p.k) else np.asarray(p.k, np.float64)
        ref = oracle.dt_max(shape=p.shape, h=p.h, k=k, u=p.u, bc=p.bc)
        with make_grid(p, dt=1e-30) as g:
            got = g.stability_dt()
            assert g.stability_dt() == got     # cached until the coefficients or faces change
        assert abs(got - ref) <= 1e-13 * ref, (case, mix, got, ref)


@pytest.mark.parametrize("case", ["all_tied", "one_far_row"])
def test_stability_dt_candidate_blocks(case):
    # the fp64 pass visits only the rows of the fp32 pass's blocks that can
    # hold the maximum, spread over the whole launch; with too many such
    # blocks every block takes its own rows again. all_tied: periodic faces
    # and one k value in every cell, so every block holds the maximum (more
    # than the spread path takes); one_far_row: one cell with the largest k
    # in a row past the first period of the fp32 pass's rows
    rng = np.random.default_rng(31)
    if case == "all_tied":
        shape = (20, 32, 32)
        k = np.full(shape[::-1], 1.3, np.float32)
        bc = [(P, 0.0)] * 6
    else:
        shape = (8, 128, 100)
        k = rng.uniform(0.5, 1.0, shape[::-1]).astype(np.float32)
        k[97, 101, 3] = 2.5        # row 97 * 128 + 101 = 12517, beyond 9728 warps
        bc = [(D, 0.0), (D, 1.0), (ZF, 0.0), (ZF, 0.0), (P, 0.0), (P, 0.0)]
    p = W.Problem(shape=shape, T0=np.zeros(shape[::-1], np.float32), k=k, bc=bc, steps=1)
    ref = oracle.dt_max(shape=shape, h=p.h, k=np.asarray(k, np.float64), u=p.u, bc=bc)
    with make_grid(p, dt=1e-30) as g:
        got = g.stability_dt()
    assert abs(got - ref) <= 1e-13 * ref, (case, got, ref)


def test_unstable_dt_rejected():
    p = _mixed_problem(0)
    with make_grid(p) as g:
        lim = g.stability_dt()
        g.set_dt(lim)   # the limit itself is allowed
        with pytest.raises(wfa.WfaError) as e:
            g.set_dt(lim * 1.001)
        assert e.value.code == -4


def test_total_heat_matches_oracle():
    for storage in (wfa.F32, wfa.BF16):
        p = _mixed_problem(1, seed=5)
        with make_grid(p, storage=storage) as g:
            g.step(7)
            T = g.read_field()
            e = g.total_heat()
        ref = oracle.total_heat(T.astype(np.float64), p.h)
        assert abs(e - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("mix", [1, 2])
def test_conservation_on_gpu(mix):
    # zero-flux / periodic faces: total heat changes only by fp32 rounding
    p = _mixed_problem(mix, shape=(48, 40, 36), seed=2)
    with make_grid(p) as g:
        e0 = g.total_heat()
        g.step(200)
        e1 = g.total_heat()
    assert abs(e1 - e0) <= 1e-5 * abs(e0)


# ------------------------------------------------------- state & errors --
def test_call_order_errors():
    g = wfa.Grid((8, 8, 8))
    with pytest.raises(wfa.WfaError) as e:
        g.step(1)
    assert e.value.code == -7
    g.set_bcs([(P, 0), (D, 0)] + [(ZF, 0)] * 4)
    g.set_coeffs(1.0)
    with pytest.raises(wfa.WfaError) as e:
        g.stability_dt()
    assert e.value.code == -3
    g.close()



def test_argument_limits():
    # edges, cell sizes, storage, faces larger than the 32-bit face kernels
    # take, values and kinds out of range: refused with WFA_ERR_ARG / _BC
    bad = [((1, 8, 8), {}), ((8, 8, 8), {"h": (1.0, 0.0, 1.0)}), ((8, 8, 8), {"h": (1.0, float("nan"), 1.0)}),
           ((8, 8, 8), {"storage": 7}), ((70000, 70000, 2), {})]
    for shape, kw in bad:
        with pytest.raises(wfa.WfaError) as e:
            wfa.Grid(shape, **kw)
        assert e.value.code == -1, (shape, kw)
    with wfa.Grid((8, 8, 8)) as g:
        for call, code in [(lambda: g.set_bc(6, ZF, 0.0), -1), (lambda: g.set_bc(0, 9, 0.0), -1),
                           (lambda: g.set_bc(0, D, float("inf")), -1), (lambda: g.set_coeffs(-1.0), -1),
                           (lambda: g.set_tuning(9, 0), -1), (lambda: g.set_tuning(1, 8), -1)]:
            with pytest.raises(wfa.WfaError) as e:
                call()
            assert e.value.code == code
        k = np.ones((8, 8, 8), np.float32)
        k[3, 4, 5] = np.nan
        with pytest.raises(wfa.WfaError) as e:
            g.set_coeffs(k)
        assert e.value.code == -1 and "k[" in str(e.value)
    with wfa.Grid((2, 8, 8)) as g:
        with pytest.raises(wfa.WfaError) as e:
            g.set_bc(0, DC, 1.0)   # a held layer needs an edge of 3
        assert e.value.code == -3


def test_injected_allocation_failures():
    # host-side fault injection: an allocation made to fail reports
    # WFA_ERR_OOM and leaves the grid as it was; nothing faults on the device
    try:
        for n in range(4):   # each of wfa_create_grid's four device buffers
            wfa.inject_alloc_failure(n)
            with pytest.raises(wfa.WfaError) as e:
                wfa.Grid((24, 20, 18))
            assert e.value.code == -2 and "out of memory" in str(e.value)
        wfa.inject_alloc_failure(-1)
        p = _mixed_problem(2, shape=(24, 20, 18), kvar=True, adv=False, seed=21)
        dt = oracle_dt(p)   # within the limits of both conductivities
        q = W.Problem(shape=p.shape, T0=p.T0, k=0.8, u=p.u, bc=p.bc, h=p.h, dt=dt, steps=4)
        with make_grid(q) as g:
            g.step(2)
            wfa.inject_alloc_failure(1)   # k is allocated, 1/k is not
            with pytest.raises(wfa.WfaError) as e:
                g.set_coeffs(p.k)
            assert e.value.code == -2
            g.step(2)                     # still the uniform-k grid
            np.testing.assert_array_equal(g.read_field(), run_gpu(q))
            g.set_coeffs(p.k)             # and per-cell k works afterwards
            g.set_dt(dt)                  # (new coefficients ask for dt again)
            g.step(3)
            ref = run_oracle(q, steps=4)
            ref = run_oracle(W.Problem(shape=p.shape, T0=ref.astype(np.float32), k=p.k, u=p.u, bc=p.bc, h=p.h,
                                       dt=dt, steps=3))
            assert rel_linf(g.read_field(), ref) <= F32_TOL
    finally:
        wfa.inject_alloc_failure(-1)
    # the same through the environment, in a fresh process: the third
    # allocation (the reduction buffer of wfa_create_grid) fails
    code = ("import paper_2209_13768_gb300 as wfa\n"
            "try:\n    wfa.Grid((8, 8, 8))\nexcept wfa.WfaError as e:\n    print('code', e.code)\n"
            "g = wfa.Grid((8, 8, 8)); g.close(); print('then ok')\n")
    env = dict(os.environ, WFA_FAULT_ALLOC_AT="3")
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "code -2" in r.stdout and "then ok" in r.stdout


def test_degenerate_coefficients():
    # k = 0 and no advection: nothing moves, the limit is infinite
    rng = np.random.default_rng(13)
    T0 = rng.random((9, 10, 11), dtype=np.float32)
    p = W.Problem(shape=(11, 10, 9), T0=T0, k=0.0, bc=[(D, 1.0)] * 6, steps=5)
    with wfa.Grid(p.shape) as g:
        g.set_bcs(p.bc)
        g.set_coeffs(0.0)
        g.set_field(T0)
        assert g.stability_dt() == float("inf")
        g.set_dt(1e6)
        g.step(5)
        np.testing.assert_array_equal(g.read_field(), T0)
    # pure advection at Courant number 1 on a periodic box: a shift by one
    # cell per step (to rounding: T + (T_up - T))
    p = W.Problem(shape=(16, 12, 10), T0=rng.random((10, 12, 16), dtype=np.float32), k=0.0, u=(1.0, 0.0, 0.0),
                  bc=[(P, 0.0)] * 6, dt=1.0, steps=3)
    T = run_gpu(p)
    np.testing.assert_allclose(T, np.roll(p.T0, 3, axis=2), rtol=0, atol=5e-7)
    # a single zero-conductivity cell insulates itself: it keeps its value
    p = _mixed_problem(1, shape=(12, 11, 10), kvar=True, adv=False, seed=3)
    k = np.asarray(p.k).copy()
    k[4, 5, 6] = 0.0
    p.k = k
    T = run_gpu(p, steps=6)
    assert T[4, 5, 6] == p.T0[4, 5, 6]
    assert rel_linf(T, run_oracle(p, steps=6)) <= F32_TOL


def test_checkpoint_resume_is_bitwise():
    p = _mixed_problem(4, seed=9)
    full = run_gpu(p, steps=23, depth=3, variant=1)
    with make_grid(p, depth=2, variant=2) as g:
        g.step(10)
        mid = g.read_field()
    q = W.Problem(shape=p.shape, T0=mid, k=p.k, u=p.u, bc=p.bc, h=p.h)
    with make_grid(q, dt=None) as g2:
        g2.set_dt(run_dt(p))
        g2.step(13)
        np.testing.assert_array_equal(g2.read_field(), full)


def run_dt(p):
    with make_grid(p) as g:
        return p.dt if p.dt else p.dt_factor * g.stability_dt()


# ------------------------------------------ reduced copies of the configs --
def test_lognormal_reduced():
    p = W.heat_lognormal(shape=(96, 80, 72), steps=100)
    ref = run_oracle(p)
    for depth in (1, 2, 4):
        T = run_gpu(p, depth=depth)
        assert rel_linf(T, ref) <= F32_TOL
        assert T.min() >= -1e-6 and T.max() <= 1 + 1e-6   # maximum principle


@pytest.mark.parametrize("storage", [wfa.F32, wfa.BF16])
def test_advection_diffusion_reduced(storage):
    p = W.advection_diffusion(shape=(128, 96, 64), steps=100)
    ref = run_oracle(p)
    T = run_gpu(p, storage=storage)
    err = rel_linf(T, ref)
    assert err <= (F32_TOL if storage == wfa.F32 else bf16_bound(p.steps)), err
    np.testing.assert_array_equal(run_gpu(p, storage=storage, depth=2, variant=4), run_gpu(p, storage=storage, variant=3))
    np.testing.assert_array_equal(run_gpu(p, storage=storage, depth=2, variant=7), run_gpu(p, storage=storage, variant=3))


def test_autotune_keeps_state_and_results():
    p = _mixed_problem(4, shape=(70, 45, 33), seed=21)
    ref = run_gpu(p, steps=17, variant=-1)
    with make_grid(p) as g:
        g.step(5)
        before = g.read_field()
        d, v = g.autotune()
        assert 1 <= d <= 8 and v in (1, 2, 3, 4, 5, 6, 7)
        np.testing.assert_array_equal(g.read_field(), before)
        assert g.steps_done() == 5
        g.step(12)
        np.testing.assert_array_equal(g.read_field(), ref)


@pytest.mark.parametrize("depth,variant", [(1, 3), (2, 1), (1, -1)])
def test_kernel_timing_samples_and_leaves_results_alone(depth, variant):
    p = W.heat_lognormal(shape=(40, 33, 27), steps=12)
    ref = run_gpu(p, depth=depth, variant=variant)
    with make_grid(p, depth=depth, variant=variant) as g:
        assert g.kernel_time() == (0.0, 0)          # off: nothing recorded
        g.set_kernel_timing(2)                       # passes 0, 2, 4, ... are sampled
        n0 = g.launch_count()
        g.step(p.steps)
        # ghost-layer faces: one kernel per pass for every variant here
        assert g.launch_count() - n0 == p.steps // depth
        ms, n = g.kernel_time()
        assert n == (p.steps // depth + 1) // 2 and ms > 0
        assert g.kernel_time() == (0.0, 0)           # a read starts a new count
        g.set_kernel_timing(0)
        np.testing.assert_array_equal(g.read_field(), ref)
        with pytest.raises(wfa.WfaError):
            g.set_kernel_timing(-1)


@pytest.mark.parametrize("depth,variant", [(1, 3), (1, 5), (2, 4), (2, 1)])
def test_small_grid_step_graphs(depth, variant):
    # small grids replay captured runs of passes; the fields must be those of
    # the same passes launched one call at a time, also after the
    # configuration changes (a stale graph would replay the old one)
    p = _mixed_problem(6, shape=(40, 24, 20), kvar=variant != 4, seed=5)
    n = 150
    with make_grid(p, depth=depth, variant=variant) as g, make_grid(p, depth=depth, variant=variant) as h:
        g.step(n)
        for _ in range(n):
            h.step(1)
        np.testing.assert_array_equal(g.read_field(), h.read_field())
        dt2 = 0.5 * g.stability_dt()
        for grid in (g, h):
            grid.set_dt(dt2)
        g.step(n + 1)
        for _ in range(n + 1):
            h.step(1)
        np.testing.assert_array_equal(g.read_field(), h.read_field())
        g.set_bc(2, D, 0.75)
        h.set_bc(2, D, 0.75)
        for grid in (g, h):
            grid.set_dt(dt2)
        g.step(2 * n)
        for _ in range(2 * n):
            h.step(1)
        np.testing.assert_array_equal(g.read_field(), h.read_field())


@pytest.mark.parametrize("storage", [wfa.F32, wfa.BF16])
def test_pinned_host_buffers_go_direct(storage):
    # pinned host memory is packed / unpacked by the kernels themselves,
    # pageable memory through the staging buffer: same fields either way
    torch = pytest.importorskip("torch")
    p = _mixed_problem(5, shape=(37, 29, 23), seed=4)
    with make_grid(p, storage=storage) as g:
        g.step(7)
        pageable = g.read_field()
        pinned = torch.empty(tuple(p.T0.shape), dtype=torch.float32).pin_memory()
        g.read_field(pinned)
        np.testing.assert_array_equal(pinned.numpy(), pageable)
        T0 = torch.from_numpy(np.ascontiguousarray(p.T0)).pin_memory()
        g.set_field(T0)
        g.step(7)
        np.testing.assert_array_equal(g.read_field(), pageable)


def test_pinned_conductivity_goes_direct():
    # pinned k is read by the checking kernel itself, pageable k through the
    # staging buffer: the same fields, and an invalid pinned k is rejected
    # with the grid left as it was
    torch = pytest.importorskip("torch")
    p = _mixed_problem(6, shape=(37, 29, 23), kvar=True, adv=True, seed=9)
    ref = run_gpu(p, steps=6)
    with make_grid(p) as g:
        kp = torch.from_numpy(np.ascontiguousarray(p.k, dtype=np.float32)).pin_memory()
        g.set_field(p.T0)
        g.set_coeffs(kp, p.u)
        g.set_dt(p.dt if p.dt else p.dt_factor * g.stability_dt())
        g.step(6)
        np.testing.assert_array_equal(g.read_field(), ref)
        bad = kp.clone().pin_memory()
        bad.view(-1)[1234] = float("nan")
        with pytest.raises(wfa.WfaError) as e:
            g.set_coeffs(bad, p.u)
        assert "1234" in str(e.value)
        g.set_field(p.T0)
        g.set_dt(p.dt if p.dt else p.dt_factor * g.stability_dt())
        g.step(6)
        np.testing.assert_array_equal(g.read_field(), ref)


def test_caller_owned_buffers():
    # fields and k in caller-owned device memory (torch tensors): the same
    # results, before and after set_coeffs, and the caller's memory is used
    torch = pytest.importorskip("torch")
    p = _mixed_problem(6, shape=(41, 30, 22), kvar=True, adv=False, seed=8)
    ref = run_gpu(p, steps=9)
    with make_grid(p) as g:
        fb, kb = g.buffer_bytes()
        Ta = torch.empty(fb, dtype=torch.uint8, device="cuda")
        Tb = torch.empty(fb, dtype=torch.uint8, device="cuda")
        k = torch.empty(kb, dtype=torch.uint8, device="cuda")
        r = torch.empty(kb, dtype=torch.uint8, device="cuda")
        g.attach_buffers(Ta, Tb, k, r)
        g.step(9)
        np.testing.assert_array_equal(g.read_field(), ref)
        assert Ta.any() and Tb.any() and k.any() and r.any()
    # attached while k is uniform: per-cell k set later lands in the caller's buffers
    with wfa.Grid(p.shape, h=p.h) as g:
        fb, kb = g.buffer_bytes()
        bufs = [torch.empty(b, dtype=torch.uint8, device="cuda") for b in (fb, fb, kb, kb)]
        g.attach_buffers(*bufs)
        g.set_bcs(p.bc)
        g.set_coeffs(p.k, p.u)
        g.set_field(p.T0)
        g.set_dt(p.dt_factor * g.stability_dt())
        g.step(9)
        np.testing.assert_array_equal(g.read_field(), ref)
        assert bufs[2].any()
    with wfa.Grid(p.shape) as g:
        with pytest.raises(wfa.WfaError):
            g.attach_buffers(Ta, Ta)


def _face_flux_ref(T, p, dt):
    """The Dirichlet face flux of one step, in fp64 from its definition."""
    T = np.asarray(T, np.float64)
    k = np.broadcast_to(np.asarray(p.k, np.float64), T.shape)
    tot = 0.0
    for f, (kind, tb) in enumerate(p.bc):
        if kind != D:
            continue
        ax, side = f // 2, f % 2
        arr_ax = 2 - ax                                   # arrays are [z, y, x]
        idx = [slice(None)] * 3
        idx[arr_ax] = -1 if side else 0
        tc, kc = T[tuple(idx)], k[tuple(idx)]
        h, u = p.h[ax], p.u[ax]
        tot += np.sum(2.0 * kc * (tb - tc) / (h * h))
        uh = u / h
        tbf = np.full(tc.shape, float(tb))
        if side == 0:
            tot += np.sum(uh * tbf if uh > 0 else uh * tc)
        else:
            tot -= np.sum(uh * tc if uh > 0 else uh * tbf)
    return tot * dt * p.h[0] * p.h[1] * p.h[2]


@pytest.mark.parametrize("kvar,adv", [(True, True), (False, True), (True, False)])
def test_boundary_flux_balances_energy(kvar, adv):
    # Dirichlet faces (one held at a value per side), zero flux and periodic
    # elsewhere: the energy change of one step is the face flux (fp64 sum,
    # fp32 step rounding)
    p = _mixed_problem(6, shape=(37, 29, 23), kvar=kvar, adv=adv, seed=12)
    with make_grid(p) as g:
        g.step(3)
        dt = p.dt_factor * g.stability_dt()
        T = g.read_field()
        e0 = g.total_heat()
        flux = g.boundary_flux()
        assert abs(flux - _face_flux_ref(T, p, dt)) <= 1e-12 * max(1.0, abs(flux)) * T.size
        g.step(1)
        e1 = g.total_heat()
        assert abs((e1 - e0) - flux) <= 2e-6 * np.abs(T).sum() * np.prod(p.h), (e1 - e0, flux)
    pdc = _mixed_problem(3)
    with make_grid(pdc) as g:
        with pytest.raises(wfa.WfaError) as e:
            g.boundary_flux()
        assert e.value.code == -3
