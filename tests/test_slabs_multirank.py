"""The slab decomposition's host-side logic on CPU ranks (gloo): how the grid
is split, which faces become exchange faces, and the exchange of boundary
planes between ranks with the fp64 reductions.

The end-to-end check runs a z-split heat solve on 2 and 3 gloo ranks: each
rank holds its slab plus one halo plane on each side, the planes move with
``exchange_halos`` before every step, and a plain numpy update of the
uniform-k 7-point step (Eq. expl_form, periodic x / y) advances the slab. The
gathered field must equal the oracle's whole-grid result, with a periodic and
with a zero-flux z axis; the all-reduced heat and stability limit must equal
the whole grid's."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2209_13768_gb300 import slabs  # noqa: E402


def test_split_covers_the_axis():
    for nz in (3, 7, 64, 513):
        for parts in range(1, min(nz, 9) + 1):
            r = slabs.split_z(nz, parts)
            assert r[0][0] == 0 and r[-1][1] == nz and len(r) == parts
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        slabs.split_z(4, 5)


def test_slab_faces():
    bc = [("dirichlet", 1.0), ("zeroflux", 0.0), ("periodic", 0.0), ("periodic", 0.0),
          ("dirichlet_cell", 0.5), ("dirichlet", 0.0)]
    assert slabs.slab_faces(bc, 0, 1) == bc
    assert slabs.slab_faces(bc, 0, 3)[4:] == [("dirichlet_cell", 0.5), ("exchange", 0.0)]
    assert slabs.slab_faces(bc, 1, 3)[4:] == [("exchange", 0.0), ("exchange", 0.0)]
    assert slabs.slab_faces(bc, 2, 3)[4:] == [("exchange", 0.0), ("dirichlet", 0.0)]
    per = bc[:4] + [("periodic", 0.0)] * 2
    for i in range(3):
        assert slabs.slab_faces(per, i, 3)[4:] == [("exchange", 0.0)] * 2
        assert slabs.slab_faces(per, i, 3)[:4] == bc[:4]
    assert slabs.neighbours(0, 3, False) == (None, 1)
    assert slabs.neighbours(2, 3, False) == (1, None)
    assert slabs.neighbours(0, 3, True) == (2, 1)
    assert slabs.neighbours(0, 1, True) == (0, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


SHAPE = (12, 10, 13)   # nx, ny, nz
W = 0.12               # k dt / h^2 (uniform k)
STEPS = 7


def _initial():
    nx, ny, nz = SHAPE
    return np.random.default_rng(77).uniform(0.0, 1.0, (nz, ny, nx))


def _numpy_step(a, w):
    """Uniform-k 7-point step of the interior planes of a (planes 1 .. -2),
    x and y periodic, z neighbours from the planes around them."""
    c = a[1:-1]
    s = (np.roll(c, 1, 2) + np.roll(c, -1, 2) + np.roll(c, 1, 1) + np.roll(c, -1, 1) + a[:-2] + a[2:])
    out = a.copy()
    out[1:-1] = c + w * (s - 6.0 * c)
    return out


def _rank_main(rank, world, port, wrap, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        T = _initial()
        z0, z1 = slabs.split_z(SHAPE[2], world)[rank]
        a = np.zeros((z1 - z0 + 2,) + T.shape[1:])
        a[1:-1] = T[z0:z1]
        t = torch.from_numpy(a)
        down, up = slabs.neighbours(rank, world, wrap)
        for _ in range(STEPS):
            slabs.exchange_halos(dist, rank, world, t[1], t[-2], t[0] if down is not None else None,
                                 t[-1] if up is not None else None, wrap)
            if down is None:      # zero-flux z face: the ghost plane mirrors the boundary plane
                t[0] = t[1]
            if up is None:
                t[-1] = t[-2]
            t.copy_(torch.from_numpy(_numpy_step(t.numpy(), W)))
        parts = [None] * world
        dist.all_gather_object(parts, (z0, t[1:-1].numpy().copy()))
        heat = slabs.allreduce_sum(dist, float(t[1:-1].sum()), "cpu")
        lim = slabs.allreduce_min(dist, [0.5, 0.25, 0.75][rank % 3], "cpu")
        if rank == 0:
            out.put((sorted(parts, key=lambda p: p[0]), heat, lim))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,wrap", [(2, True), (2, False), (3, True), (3, False)])
def test_distributed_slab_solve_matches_oracle(world, wrap):
    import oracle
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, wrap, out)) for r in range(world)]
    for p in procs:
        p.start()
    parts, heat, lim = out.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([p[1] for p in parts], axis=0)
    zbc = ("periodic", 0.0) if wrap else ("zeroflux", 0.0)
    bc = [("periodic", 0.0)] * 4 + [zbc, zbc]
    ref = oracle.run(_initial(), STEPS, shape=SHAPE, k=W, bc=bc, dt=1.0)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    assert heat == pytest.approx(oracle.total_heat(ref), rel=1e-13)
    assert lim == 0.25 if world >= 2 else 0.5
