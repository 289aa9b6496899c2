"""One grid split into slabs along z (exchange faces), on one GPU: the
slabs' field is bitwise the undivided grid's for every boundary mix, per-cell
and uniform k, advection, fp32 and bf16, uneven slabs and a single wrapping
slab; the slab stability limits and heat add up to the whole grid's; the
calls that cannot take exchange faces refuse them."""
import numpy as np
import pytest

import paper_2209_13768_gb300 as wfa
from paper_2209_13768_gb300 import slabs
from paper_2209_13768_gb300 import workloads as W

pytestmark = pytest.mark.gpu

D, ZF, P, DC = W.D, W.ZF, W.P, W.DC
MIXES = [
    [(D, 0.3), (D, -0.7), (D, 1.0), (D, 0.0), (D, 0.5), (D, 2.0)],
    [(ZF, 0)] * 6,
    [(P, 0)] * 6,
    [(DC, 0.25), (DC, 0.75), (DC, -0.5), (DC, 1.0), (DC, 0.1), (DC, 0.2)],
    [(D, 1.0), (ZF, 0), (P, 0), (P, 0), (DC, 0.5), (D, 0.0)],
    [(DC, 1.0), (D, 0.0), (ZF, 0), (DC, 0.3), (P, 0), (P, 0)],
    [(P, 0), (P, 0), (D, 0.2), (ZF, 0), (ZF, 0), (D, 0.8)],
]


def _problem(mix, shape=(37, 29, 23), kvar=True, adv=True, seed=0):
    rng = np.random.default_rng(2000 + seed)
    nx, ny, nz = shape
    k = np.exp(0.5 * rng.standard_normal((nz, ny, nx))).astype(np.float32) if kvar else 0.8
    u = tuple(rng.uniform(-0.4, 0.4, 3)) if adv else (0.0, 0.0, 0.0)
    h = tuple(rng.uniform(0.8, 1.25, 3))
    T0 = rng.uniform(0, 1, (nz, ny, nx)).astype(np.float32)
    return W.Problem(shape=shape, T0=T0, k=k, u=u, bc=MIXES[mix], h=h, steps=15)


def _whole(p, storage, dt, variant=3):
    with wfa.Grid(p.shape, h=p.h, storage=storage) as g:
        g.set_bcs(p.bc)
        g.set_coeffs(p.k, p.u)
        g.set_field(p.T0)
        g.set_dt(dt)
        g.set_tuning(1, variant)
        g.step(p.steps)
        return g.read_field(), g.total_heat()


def _dt(p, storage=wfa.F32):
    with wfa.Grid(p.shape, h=p.h, storage=storage) as g:
        g.set_bcs(p.bc)
        g.set_coeffs(p.k, p.u)
        return g.stability_dt()


@pytest.mark.parametrize("kvar,adv", [(True, True), (False, True), (True, False), (False, False)])
@pytest.mark.parametrize("mix", range(len(MIXES)))
def test_slabs_bitwise_equal_whole_grid(mix, kvar, adv):
    p = _problem(mix, kvar=kvar, adv=adv, seed=mix)
    dt_whole = _dt(p)
    dt = 0.9 * dt_whole
    ref, heat = _whole(p, wfa.F32, dt)
    for parts in (2, 3, 4):
        with slabs.SlabGrid(p.shape, parts, h=p.h, bc=p.bc) as s:
            s.set_coeffs(p.k, p.u)
            assert s.stability_dt() == dt_whole, parts   # the same fp64 maximum over the same cells
            s.set_field(p.T0)
            s.set_dt(dt)
            for variant in (3, 5):
                s.set_field(p.T0)
                s.set_tuning(1, variant)
                s.step(p.steps)
                np.testing.assert_array_equal(s.read_field(), ref, err_msg=f"{parts} slabs, variant {variant}")
            assert s.total_heat() == pytest.approx(heat, rel=1e-12, abs=1e-9)


@pytest.mark.parametrize("mix", [0, 3, 5])
def test_slabs_on_their_own_streams(mix):
    """Each slab on its own stream: the exchanges order the streams."""
    torch = pytest.importorskip("torch")
    p = _problem(mix, kvar=mix != 3, adv=True, seed=20 + mix)
    dt = 0.9 * _dt(p)
    ref, _ = _whole(p, wfa.F32, dt)
    streams = [torch.cuda.Stream() for _ in range(3)]
    with slabs.SlabGrid(p.shape, 3, h=p.h, bc=p.bc, streams=[s.cuda_stream for s in streams]) as s:
        s.set_coeffs(p.k, p.u)
        s.set_field(p.T0)
        s.set_dt(dt)
        s.set_tuning(1, 3)
        s.step(p.steps)
        s.sync()
        np.testing.assert_array_equal(s.read_field(), ref)


@pytest.mark.parametrize("mix", [0, 2, 4, 6])
def test_slabs_bf16(mix):
    p = _problem(mix, kvar=True, adv=True, seed=10 + mix)
    dt = 0.9 * _dt(p, wfa.BF16)
    ref, _ = _whole(p, wfa.BF16, dt)
    with slabs.SlabGrid(p.shape, 3, h=p.h, storage=wfa.BF16, bc=p.bc) as s:
        s.set_coeffs(p.k, p.u)
        s.set_field(p.T0)
        s.set_dt(dt)
        s.step(p.steps)
        np.testing.assert_array_equal(s.read_field(), ref)


def test_uneven_and_chunked_slabs_and_calls_in_pieces():
    """Slabs of 3, 10 and 10 planes, the column kernel with several z chunk
    lengths, and a run split over several calls."""
    p = _problem(4, shape=(40, 21, 23), seed=3)
    dt = 0.9 * _dt(p)
    ref, _ = _whole(p, wfa.F32, dt)
    with slabs.SlabGrid(p.shape, 3, h=p.h, bc=p.bc) as s:
        s.ranges = [(0, 3), (3, 13), (13, 23)]
        s.close()
        s.slabs = [wfa.Grid((40, 21, z1 - z0), h=p.h) for z0, z1 in s.ranges]
        s.set_bcs(p.bc)
        s.set_coeffs(p.k, p.u)
        s.set_dt(dt)
        for zc in (0, 1, 2, 4):
            for g in s.slabs:
                g.set_zchunk(zc)
            s.set_field(p.T0)
            s.step(4)
            s.step(0)
            s.step(p.steps - 4)
            np.testing.assert_array_equal(s.read_field(), ref, err_msg=f"zchunk {zc}")


def test_single_wrapping_slab_equals_periodic_grid():
    p = _problem(2, shape=(33, 17, 19), seed=5)     # all periodic
    dt = 0.9 * _dt(p)
    ref, _ = _whole(p, wfa.F32, dt)
    with slabs.SlabGrid(p.shape, 1, h=p.h, bc=p.bc) as s:
        assert s.slabs[0] is not None
        s.set_coeffs(p.k, p.u)
        s.set_field(p.T0)
        s.set_dt(dt)
        s.step(p.steps)
        np.testing.assert_array_equal(s.read_field(), ref)


def test_exchange_faces_are_refused_where_they_cannot_work():
    p = _problem(0, shape=(20, 18, 16), adv=False, seed=7)
    with slabs.SlabGrid(p.shape, 2, h=p.h, bc=p.bc) as s:
        s.set_coeffs(p.k, p.u)
        s.set_field(p.T0)
        s.set_dt(0.5 * s.stability_dt())
        with pytest.raises(wfa.WfaError) as e:
            wfa.batch_run(s.slabs, [2, 2])
        assert e.value.code == -3
        with pytest.raises(wfa.WfaError) as e:
            s.slabs[0].implicit_step(0.1, 1)
        assert e.value.code == -3
        with pytest.raises(wfa.WfaError):
            wfa.slabs_step(s.slabs[::-1], 1)          # out of order: faces do not meet
        with pytest.raises(wfa.WfaError):
            s.slabs[0].exchange_planes(wfa.ZLO)        # the real -z face is not an exchange face
        snd, rcv, nb = s.slabs[0].exchange_planes(wfa.ZHI)
        assert snd and rcv and nb > 0 and rcv - snd == nb   # the halo plane follows the last own plane
    with wfa.Grid((8, 8, 8)) as g:
        with pytest.raises(wfa.WfaError) as e:
            g.set_bc(0, "exchange")                   # x faces cannot be exchange faces
        assert e.value.code == -3


def test_tiled_kernels_fall_back_to_the_column_kernel_on_slabs():
    p = _problem(1, shape=(36, 20, 18), seed=9)
    dt = 0.9 * _dt(p)
    ref, _ = _whole(p, wfa.F32, dt)
    with slabs.SlabGrid(p.shape, 2, h=p.h, bc=p.bc) as s:
        s.set_coeffs(p.k, p.u)
        s.set_field(p.T0)
        s.set_dt(dt)
        s.set_tuning(4, 1)                            # asks for the tiled kernel, depth 4
        assert s.slabs[0].tuning()[:2] == (1, 3)
        s.step(p.steps)
        np.testing.assert_array_equal(s.read_field(), ref)
