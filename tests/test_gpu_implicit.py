"""GPU parity of the implicit step (backward Euler solved by classic CG,
Sec. 1.1.2, Eq. impl_form) against the FP64 oracle.

Tolerances. The GPU iterates in fp32 with fp64 inner products and stops on
its recursively updated residual; the oracle runs the same CG in fp64 to
1e-12. With rtol = 1e-7 the GPU solution differs from the exact one by the
fp32 floor of the residual (about 1e-7 ||b||) times the condition number of
A = I + dt L, at most 1 + dt * 12 k_max / h_min^2 (~15 for the cases below),
plus the fp32 rounding of the field itself; 3e-5 relative to max |T|
covers three steps with a margin. Fixed iteration counts (rtol = 0) compare
the CG iterates themselves: fp32 rounding of each product, amplified by no
more than the same condition number, stays below 1e-5.
"""
import os

import numpy as np
import pytest

import oracle
import paper_2209_13768_gb300 as wfa
from paper_2209_13768_gb300 import workloads as W
from helpers import rel_linf

pytestmark = pytest.mark.gpu

D, ZF, P, DC = W.D, W.ZF, W.P, W.DC
TOL = 3e-5

MIXES = [
    [(D, 0.3), (D, -0.7), (D, 1.0), (D, 0.0), (D, 0.5), (D, 2.0)],
    [(ZF, 0)] * 6,
    [(P, 0)] * 6,
    [(DC, 0.25), (DC, 0.75), (DC, -0.5), (DC, 1.0), (DC, 0.1), (DC, 0.2)],
    [(D, 1.0), (ZF, 0), (P, 0), (P, 0), (DC, 0.5), (D, 0.0)],
    [(DC, 1.0), (D, 0.0), (ZF, 0), (DC, 0.3), (P, 0), (P, 0)],
    [(P, 0), (P, 0), (D, 0.2), (ZF, 0), (ZF, 0), (D, 0.8)],
]


def _problem(mix, shape=(37, 29, 23), kvar=True, seed=0):
    rng = np.random.default_rng(2000 + seed)
    nx, ny, nz = shape
    k = np.exp(0.5 * rng.standard_normal((nz, ny, nx))).astype(np.float32) if kvar else 0.8
    h = tuple(rng.uniform(0.8, 1.25, 3))
    T0 = rng.uniform(0, 1, (nz, ny, nx)).astype(np.float32)
    return W.Problem(shape=shape, T0=T0, k=k, bc=MIXES[mix], h=h)


def _dt(p, factor=5.0):
    """factor x the explicit step's stability limit (backward Euler has none)."""
    kk = p.k if np.isscalar(p.k) else np.asarray(p.k, dtype=np.float64)
    return factor * oracle.dt_max(shape=p.shape, h=p.h, k=kk, bc=p.bc)


def _grid(p):
    g = wfa.Grid(p.shape, h=p.h)
    g.set_bcs(p.bc)
    g.set_coeffs(p.k)
    g.set_field(p.T0)
    return g


def _oracle(p, steps, dt, rtol=1e-12, max_iter=10000):
    kk = p.k if np.isscalar(p.k) else np.asarray(p.k, dtype=np.float64)
    return oracle.implicit(p.T0, steps, shape=p.shape, h=p.h, k=kk, bc=p.bc, dt=dt, rtol=rtol, max_iter=max_iter)


@pytest.mark.parametrize("kvar", [False, True])
@pytest.mark.parametrize("mix", range(len(MIXES)))
def test_implicit_matches_oracle(mix, kvar):
    p = _problem(mix, kvar=kvar, seed=mix)
    dt = _dt(p)
    ref, _, _ = _oracle(p, 3, dt)
    with _grid(p) as g:
        iters, res = g.implicit_step(dt, 3, rtol=1e-7, max_iter=500)
        T = g.read_field()
        assert g.steps_done() == 3
    assert 0 < iters < 3 * 500 and res <= 1e-7
    assert rel_linf(T, ref) <= TOL


@pytest.mark.parametrize("kvar", [False, True])
@pytest.mark.parametrize("mix", [0, 3, 4, 5])
def test_implicit_fixed_iterations_match_oracle_iterates(mix, kvar):
    # rtol = 0: exactly m CG iterations on both sides, so the iterates
    # themselves are compared (not just the converged solution)
    p = _problem(mix, kvar=kvar, seed=10 + mix)
    dt = _dt(p, 3.0)
    for m in (1, 2, 5, 9):
        ref, it_ref, _ = _oracle(p, 1, dt, rtol=0.0, max_iter=m)
        with _grid(p) as g:
            iters, _ = g.implicit_step(dt, 1, rtol=0.0, max_iter=m)
            T = g.read_field()
        assert iters == it_ref == m
        assert rel_linf(T, ref) <= 1e-5, m


def test_implicit_iteration_counts_match_oracle():
    for mix, kvar in [(0, False), (3, True), (5, True), (6, False)]:
        p = _problem(mix, kvar=kvar, seed=20 + mix)
        dt = _dt(p)
        _, it_ref, _ = _oracle(p, 1, dt, rtol=1e-4)
        with _grid(p) as g:
            iters, res = g.implicit_step(dt, 1, rtol=1e-4)
        assert abs(iters - it_ref) <= 1 and res <= 1e-4


@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 5, 7), (64, 16, 3), (65, 17, 9), (130, 33, 20)])
def test_implicit_small_and_ragged_shapes(shape):
    for mix in (0, 4, 5, 6):
        if any(kind == DC and shape[f // 2] < 3 for f, (kind, _) in enumerate(MIXES[mix])):
            continue   # a held layer needs an edge of at least 3 cells
        for kvar in (False, True):
            p = _problem(mix, shape=shape, kvar=kvar, seed=mix + shape[0])
            dt = _dt(p, 4.0)
            ref, _, _ = _oracle(p, 2, dt)
            with _grid(p) as g:
                g.implicit_step(dt, 2, rtol=1e-7, max_iter=400)
                T = g.read_field()
            assert rel_linf(T, ref) <= TOL, (shape, mix, kvar)


def test_implicit_single_mode_one_iteration():
    # an eigenmode of the uniform-k operator: r0 is an eigenvector of A, so
    # CG needs one iteration a step and the mode is divided by 1 + dt rate
    shape = (48, 40, 24)
    nx, ny, nz = shape
    kval, dt = 0.7, 0.8
    i = np.arange(nx) + 0.5
    j = np.arange(ny)
    l = np.arange(nz)
    vx, lx = np.sin(np.pi * 2 * i / nx), 4 * np.sin(np.pi * 2 / (2 * nx)) ** 2      # Dirichlet faces, m = 2
    vy, ly = np.cos(2 * np.pi * 3 * j / ny), 4 * np.sin(np.pi * 3 / ny) ** 2       # periodic, m = 3
    vz, lz = np.sin(np.pi * 1 * l / (nz - 1)), 4 * np.sin(np.pi / (2 * (nz - 1))) ** 2  # held layers at 0, m = 1
    T0 = np.einsum("z,y,x->zyx", vz, vy, vx).astype(np.float32)
    bc = [(D, 0.0), (D, 0.0), (P, 0), (P, 0), (DC, 0.0), (DC, 0.0)]
    rate = kval * (lx + ly + lz)
    with wfa.Grid(shape) as g:
        g.set_bcs(bc)
        g.set_coeffs(kval)
        g.set_field(T0)
        iters, res = g.implicit_step(dt, 3, rtol=5e-5)
        T = g.read_field()
    # in fp32 the mode is an eigenvector only to rounding: the residual left
    # after the one iteration grows from step to step (about 4e-7, 2e-6, 7e-6
    # of ||b|| in a plain fp32 emulation), so three steps stay within 5e-5
    assert iters == 3 and res <= 5e-5
    np.testing.assert_allclose(T, T0.astype(np.float64) / (1 + dt * rate) ** 3, rtol=0, atol=2e-6)


@pytest.mark.parametrize("mix", [1, 2])
def test_implicit_conserves_heat(mix):
    p = _problem(mix, shape=(70, 45, 33), kvar=True, seed=40 + mix)
    with _grid(p) as g:
        E0 = g.total_heat()
        g.implicit_step(_dt(p, 20.0), 5, rtol=1e-7)
        E1 = g.total_heat()
    assert abs(E1 - E0) <= 2e-6 * abs(E0)


def test_implicit_then_explicit_steps():
    # implicit steps leave the grid ready for explicit steps (halo copies and
    # held layers rebuilt) and count in steps_done
    p = _problem(4, kvar=True, seed=50)
    dt_i = _dt(p, 6.0)
    mid, _, _ = _oracle(p, 2, dt_i)
    kk = np.asarray(p.k, dtype=np.float64)
    dt_e = 0.9 * oracle.dt_max(shape=p.shape, h=p.h, k=kk, bc=p.bc)
    ref = oracle.run(mid, 4, shape=p.shape, h=p.h, k=kk, bc=p.bc, dt=dt_e)
    with _grid(p) as g:
        g.implicit_step(dt_i, 2, rtol=1e-7)
        g.set_dt(dt_e)
        g.step(4)
        assert g.steps_done() == 6
        T = g.read_field()
        again, _ = g.implicit_step(dt_i, 1, rtol=1e-7)   # and back
        assert again > 0
    assert rel_linf(T, ref) <= TOL


def test_implicit_degenerate_and_errors():
    rng = np.random.default_rng(60)
    T0 = rng.uniform(0, 1, (9, 10, 11)).astype(np.float32)
    bc = [(DC, 0.5), (D, 0.0)] + [(ZF, 0)] * 4
    with wfa.Grid((11, 10, 9)) as g:
        g.set_bcs(bc)
        g.set_coeffs(1.0)
        g.set_field(T0)
        held = g.read_field()
        assert g.implicit_step(0.3, 0) == (0, 0.0)          # no steps
        np.testing.assert_array_equal(g.read_field(), held)
        iters, _ = g.implicit_step(0.0, 2)                  # dt = 0: r = 0, nothing to do
        assert iters == 0
        np.testing.assert_array_equal(g.read_field(), held)
        iters, _ = g.implicit_step(0.3, 1, rtol=0.0, max_iter=0)   # no iterations allowed
        assert iters == 0
        np.testing.assert_array_equal(g.read_field(), held)
        for call in (lambda: g.implicit_step(-1.0, 1), lambda: g.implicit_step(0.1, -1),
                     lambda: g.implicit_step(0.1, 1, rtol=-1.0), lambda: g.implicit_step(0.1, 1, max_iter=-1),
                     lambda: g.implicit_step(float("nan"), 1)):
            with pytest.raises(wfa.WfaError) as e:
                call()
            assert e.value.code == -1
        g.set_coeffs(1.0, (0.1, 0.0, 0.0))
        with pytest.raises(wfa.WfaError) as e:
            g.implicit_step(0.1, 1)                          # advection: not symmetric
        assert e.value.code == -1
    with wfa.Grid((8, 8, 8), storage=wfa.BF16) as g:
        g.set_coeffs(1.0)
        g.set_field(np.zeros((8, 8, 8), np.float32))
        with pytest.raises(wfa.WfaError) as e:
            g.implicit_step(0.1, 1)
        assert e.value.code == -1
    with wfa.Grid((8, 8, 8)) as g:
        with pytest.raises(wfa.WfaError) as e:
            g.implicit_step(0.1, 1)
        assert e.value.code == -7


def test_implicit_paper_workload_residual_at_full_size():
    # the benchmark's implicit workload at full size (512^3, uniform k,
    # held layers, omega = 1/10): after one step the true residual of
    # Eq. impl_form, recomputed in fp64 at sampled cells from the fields,
    # is within the fp32 floor of the solver's tolerance
    shape = W.IMPLICIT_SHAPE
    p = W.implicit_problem(shape)
    omega = p.dt
    with _grid(p) as g:
        iters, res = g.implicit_step(omega, 1, rtol=1e-6)
        T1 = g.read_field().astype(np.float64)
    assert 0 < iters < 100 and res <= 1e-6
    T0 = p.T0.astype(np.float64)
    nz, ny, nx = T0.shape
    rng = np.random.default_rng(70)
    z = rng.integers(1, nz - 1, 200000)
    y = rng.integers(1, ny - 1, 200000)
    x = rng.integers(1, nx - 1, 200000)
    nb = (T1[z, y, x - 1] + T1[z, y, x + 1] + T1[z, y - 1, x] + T1[z, y + 1, x] + T1[z - 1, y, x] + T1[z + 1, y, x])
    resid = (1 + 6 * omega) * T1[z, y, x] - omega * nb - T0[z, y, x]
    assert np.abs(resid).max() <= 2e-5 * np.abs(T0).max()
    # held layers untouched (-x at 1 away from the other held faces)
    np.testing.assert_array_equal(T1[1:-1, 1:-1, 0], p.bc[0][1])


@pytest.mark.parametrize("kvar", [False, True])
def test_implicit_shared_memory_spmv_is_bitwise_equal(kvar):
    # cg_spmv_sm (x / y neighbours of p through shared memory) runs the same
    # per-cell arithmetic and the same inner-product order as cg_spmv
    shapes = [(37, 29, 23), (65, 17, 9), (130, 33, 20), (3, 5, 7)]
    for mix in (0, 2, 4, 5):
        for shape in shapes:
            if any(kind == DC and shape[f // 2] < 3 for f, (kind, _) in enumerate(MIXES[mix])):
                continue
            p = _problem(mix, shape=shape, kvar=kvar, seed=70 + mix)
            dt = _dt(p, 4.0)
            out = {}
            for kind in ("l1", "sm"):
                os.environ["WFA_CG_SPMV"] = kind
                try:
                    with _grid(p) as g:
                        it, _ = g.implicit_step(dt, 2, rtol=1e-7, max_iter=300)
                        out[kind] = (it, g.read_field())
                finally:
                    os.environ.pop("WFA_CG_SPMV", None)
            assert out["l1"][0] == out["sm"][0], (mix, shape)
            np.testing.assert_array_equal(out["l1"][1], out["sm"][1], err_msg=f"{mix} {shape}")


# ---------------------------------------------------------------------------
# pipelined (Chronopoulos-Gear) CG: one kernel and one reduction an iteration
# ---------------------------------------------------------------------------
def _pgrid(p):
    g = _grid(p)
    g.set_cg_method("pipelined")
    return g


@pytest.mark.parametrize("kvar", [False, True])
@pytest.mark.parametrize("mix", range(len(MIXES)))
def test_pipelined_matches_oracle(mix, kvar):
    p = _problem(mix, kvar=kvar, seed=80 + mix)
    dt = _dt(p)
    ref, _, _ = _oracle(p, 3, dt)
    with _pgrid(p) as g:
        iters, res = g.implicit_step(dt, 3, rtol=1e-7, max_iter=500)
        T = g.read_field()
        assert g.steps_done() == 3
    assert 0 < iters < 1500 and res <= 1e-7
    assert rel_linf(T, ref) <= TOL


@pytest.mark.parametrize("kvar", [False, True])
@pytest.mark.parametrize("mix", [0, 2, 4, 5])
def test_pipelined_fixed_iterations_match_oracle_iterates(mix, kvar):
    # the pipelined iterates are classic CG's in exact arithmetic: compare
    # them with the oracle's Chronopoulos-Gear and classic iterates
    p = _problem(mix, kvar=kvar, seed=90 + mix)
    dt = _dt(p, 3.0)
    for m in (1, 2, 5, 9):
        ref, it_ref, _ = _oracle(p, 1, dt, rtol=0.0, max_iter=m)
        kk = p.k if np.isscalar(p.k) else np.asarray(p.k, dtype=np.float64)
        ref2, _, _ = oracle.implicit(p.T0, 1, shape=p.shape, h=p.h, k=kk, bc=p.bc, dt=dt, rtol=0.0, max_iter=m,
                                     method="cgcg")
        with _pgrid(p) as g:
            iters, _ = g.implicit_step(dt, 1, rtol=0.0, max_iter=m)
            T = g.read_field()
        assert iters == it_ref == m
        assert rel_linf(T, ref) <= 1e-5, m
        assert rel_linf(T, ref2) <= 1e-5, m


@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 5, 7), (65, 17, 9), (130, 33, 20)])
def test_pipelined_small_and_ragged_shapes(shape):
    for mix in (0, 2, 4, 5, 6):
        if any(kind == DC and shape[f // 2] < 3 for f, (kind, _) in enumerate(MIXES[mix])):
            continue
        for kvar in (False, True):
            p = _problem(mix, shape=shape, kvar=kvar, seed=mix + shape[1])
            dt = _dt(p, 4.0)
            ref, _, _ = _oracle(p, 2, dt)
            with _pgrid(p) as g:
                g.implicit_step(dt, 2, rtol=1e-7, max_iter=400)
                T = g.read_field()
            assert rel_linf(T, ref) <= TOL, (shape, mix, kvar)


def test_pipelined_iteration_counts_and_switching():
    p = _problem(4, kvar=True, seed=95)
    dt = _dt(p)
    kk = np.asarray(p.k, dtype=np.float64)
    _, it_ref, _ = oracle.implicit(p.T0, 1, shape=p.shape, h=p.h, k=kk, bc=p.bc, dt=dt, rtol=1e-4, method="cgcg")
    with _pgrid(p) as g:
        it_p, res = g.implicit_step(dt, 1, rtol=1e-4)
        assert abs(it_p - it_ref) <= 1 and res <= 1e-4
    with _pgrid(p) as g:
        g.implicit_step(dt, 1, rtol=1e-7)
        g.set_cg_method("classic")   # switching back and forth on one grid
        g.implicit_step(dt, 1, rtol=1e-7)
        g.set_cg_method("pipelined")
        g.implicit_step(dt, 1, rtol=1e-7)
        T = g.read_field()
        with pytest.raises(wfa.WfaError) as e:
            g.set_cg_method(7)
        assert e.value.code == -1
    ref, _, _ = _oracle(p, 3, dt)
    assert rel_linf(T, ref) <= TOL


def test_pipelined_conserves_heat():
    p = _problem(2, shape=(70, 45, 33), kvar=True, seed=96)
    with _pgrid(p) as g:
        E0 = g.total_heat()
        g.implicit_step(_dt(p, 20.0), 5, rtol=1e-7)
        E1 = g.total_heat()
    assert abs(E1 - E0) <= 2e-6 * abs(E0)


@pytest.mark.parametrize("method", ["classic", "pipelined"])
def test_device_loop_equals_host_loop(method):
    # the whole call as one graph (conditional loops over steps and
    # iterations) runs the same kernels in the same order as the host-checked
    # runs: identical fields and iteration counts
    for mix, kvar, shape in [(4, True, (37, 29, 23)), (2, False, (65, 17, 9)), (5, True, (3, 5, 7))]:
        p = _problem(mix, shape=shape, kvar=kvar, seed=120 + mix)
        dt = _dt(p, 4.0)
        out = {}
        for loop in ("host", "device"):
            if loop == "host":
                os.environ["WFA_CG_LOOP"] = "host"
            try:
                with _grid(p) as g:
                    g.set_cg_method(method)
                    n0 = g.launch_count()
                    it, res = g.implicit_step(dt, 3, rtol=1e-7, max_iter=300)
                    it2, _ = g.implicit_step(dt, 2, rtol=1e-6, max_iter=7)   # new parameters: rebuilt
                    out[loop] = (it, it2, res, g.read_field(), g.steps_done(), g.launch_count() - n0)
            finally:
                os.environ.pop("WFA_CG_LOOP", None)
        assert out["host"][:3] == out["device"][:3], (mix, shape)
        assert out["device"][4] == 5
        np.testing.assert_array_equal(out["host"][3], out["device"][3])
        # the device loop ran (its launch count has no converged no-op runs):
        # per step cg_init, [cg_spmv,] two control kernels; per iteration the
        # solver kernels and one control kernel
        its = out["device"][0] + out["device"][1]
        expect = 5 * 3 + 3 * its if method == "classic" else 5 * 4 + 2 * its
        assert out["device"][5] == expect, (out["device"][5], expect)
