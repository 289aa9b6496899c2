"""One grid split into slabs along z (domain decomposition: Sec. 1, Fig. 1b;
each WSE tile's 1 x 1 x Z column, Sec. 2.1, receives its neighbours' values
for every product, Sec. 3; the step time model of Eq. iteration_time_model).

Two forms, both over the C ABI's exchange faces (``WFA_BC_EXCHANGE``):

* ``SlabGrid``: all slabs on one device; ``wfa_slabs_step`` copies the
  boundary planes between slabs before every step.
* ``DistSlab``: one slab per process (a ``torch.distributed`` rank, one GPU
  each); the boundary planes move by point-to-point send / receive straight
  into the receiving slab's halo plane (NCCL between GPUs), and the stability
  limit and total heat are all-reduced in fp64.

``exchange_halos`` and the reductions are plain ``torch.distributed`` code on
tensors, so the CPU tests run them on gloo ranks with CPU tensors.
This module only arranges calls: every cell update runs in the library.
"""
from __future__ import annotations

import numpy as np

from . import EXCHANGE, PLANES_FIELD, PLANES_K, PLANES_RECIP_K, ZHI, ZLO, F32, Grid, slabs_step


def split_z(nz, parts):
    """[(z0, z1), ...]: `parts` consecutive slabs covering [0, nz), sizes
    differing by at most one plane (the larger ones first)."""
    if parts < 1 or parts > nz:
        raise ValueError(f"cannot split {nz} planes into {parts} slabs")
    base, extra = divmod(nz, parts)
    out, z = [], 0
    for i in range(parts):
        n = base + (1 if i < extra else 0)
        out.append((z, z + n))
        z += n
    return out


def slab_faces(bc, index, parts):
    """Faces of slab `index` of `parts`: the whole grid's x / y faces, its z
    faces at the ends of the z axis, exchange faces between slabs (and at
    both ends when the z axis is periodic)."""
    faces = list(bc[:4])
    wrap = bc[4][0] == "periodic"
    lo = ("exchange", 0.0) if (index > 0 or wrap) else bc[4]
    hi = ("exchange", 0.0) if (index < parts - 1 or wrap) else bc[5]
    return faces + [lo, hi]


class SlabGrid:
    """A grid of shape (nx, ny, nz) held as `parts` slabs on one device.

    Arrays are [z, y, x] as for ``Grid``; results are bitwise those of one
    ``Grid`` of the same shape (the slabs see the same operands).
    stream: one CUDA stream for every slab, or `streams`: one per slab (the
    slabs' kernels then overlap; the plane copies wait for both sides)."""

    def __init__(self, shape, parts, h=(1.0, 1.0, 1.0), storage=F32, stream=None, bc=None, streams=None):
        self.shape = tuple(int(s) for s in shape)
        self.ranges = split_z(self.shape[2], parts)
        self.bc = list(bc) if bc else [("zeroflux", 0.0)] * 6
        streams = list(streams) if streams else [stream] * parts
        if len(streams) != parts:
            raise ValueError("one stream per slab")
        self.slabs = [Grid((self.shape[0], self.shape[1], z1 - z0), h=h, storage=storage, stream=st)
                      for (z0, z1), st in zip(self.ranges, streams)]
        self.set_bcs(self.bc)

    def close(self):
        for g in self.slabs:
            g.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_bcs(self, bc):
        self.bc = list(bc)
        for i, g in enumerate(self.slabs):
            g.set_bcs(slab_faces(self.bc, i, len(self.slabs)))

    def _parts(self, a):
        return [np.ascontiguousarray(a[z0:z1]) for z0, z1 in self.ranges]

    def set_field(self, T):
        for g, part in zip(self.slabs, self._parts(np.asarray(T, dtype=np.float32))):
            g.set_field(part)

    def set_coeffs(self, k=1.0, u=(0.0, 0.0, 0.0)):
        if np.isscalar(k):
            for g in self.slabs:
                g.set_coeffs(k, u)
        else:
            for g, part in zip(self.slabs, self._parts(np.asarray(k, dtype=np.float32))):
                g.set_coeffs(part, u)
        self._exchange_k()

    def _exchange_k(self):
        from . import exchange
        n = len(self.slabs)
        for i in range(n - 1):
            exchange(self.slabs[i], self.slabs[i + 1], PLANES_K)
        if self.bc[4][0] == "periodic":
            exchange(self.slabs[-1], self.slabs[0], PLANES_K)

    def stability_dt(self):
        """The whole grid's limit: the smallest slab limit (exchange faces
        count as interior faces, with the neighbour's conductivity)."""
        return min(g.stability_dt() for g in self.slabs)

    def set_dt(self, dt):
        for g in self.slabs:
            g.set_dt(dt)

    def set_tuning(self, depth=0, variant=0):
        for g in self.slabs:
            g.set_tuning(depth, variant)

    def step(self, n):
        slabs_step(self.slabs, n)

    def sync(self):
        for g in self.slabs:
            g.sync()

    def read_field(self):
        return np.concatenate([g.read_field() for g in self.slabs], axis=0)

    def total_heat(self):
        return float(sum(g.total_heat() for g in self.slabs))


# ------------------------------------------------------------ one slab a rank --
def neighbours(rank, world, wrap):
    """(rank below, rank above) in z; None at an end of a non-periodic axis."""
    down = rank - 1 if rank > 0 else (world - 1 if wrap else None)
    up = rank + 1 if rank < world - 1 else (0 if wrap else None)
    return down, up


def exchange_halos(dist, rank, world, send_lo, send_hi, recv_lo, recv_hi, wrap):
    """Move boundary planes between the slabs of neighbouring ranks.

    send_lo / send_hi: this rank's own bottom / top plane; recv_lo / recv_hi:
    its halo planes below / above, where the neighbours' top / bottom planes
    go (None where there is no neighbour). Two phases, each one batch of
    point-to-point operations: first every top plane moves up, then every
    bottom plane moves down, so the transfers between two ranks match in
    order even when they are neighbours on both sides (two ranks, periodic).
    One rank with a periodic axis exchanges with itself (local copies)."""
    down, up = neighbours(rank, world, wrap)
    if world == 1:
        if wrap:
            recv_lo.copy_(send_hi)
            recv_hi.copy_(send_lo)
        return
    for send, send_to, recv, recv_from in ((send_hi, up, recv_lo, down), (send_lo, down, recv_hi, up)):
        ops = []
        if send_to is not None:
            ops.append(dist.P2POp(dist.isend, send, send_to))
        if recv_from is not None:
            ops.append(dist.P2POp(dist.irecv, recv, recv_from))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()


def allreduce_min(dist, value, device):
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return float(t.item())


def allreduce_sum(dist, value, device):
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class _DevicePlane:
    """A device address range seen as a uint8 CUDA array (for torch.as_tensor)."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def plane_tensor(ptr, nbytes, device):
    import torch
    return torch.as_tensor(_DevicePlane(ptr, nbytes), device=device)


class DistSlab:
    """This rank's slab of a grid split along z over `world` ranks (one GPU
    each). The slab's grid runs on torch's current stream of its device, so
    the point-to-point transfers (queued by torch.distributed on that stream's
    order) and the library's kernels are ordered without a host wait."""

    def __init__(self, dist, shape, rank, world, h=(1.0, 1.0, 1.0), storage=F32, bc=None):
        import torch
        self.dist, self.rank, self.world = dist, rank, world
        self.shape = tuple(int(s) for s in shape)
        self.z0, self.z1 = split_z(self.shape[2], world)[rank]
        self.bc = list(bc) if bc else [("zeroflux", 0.0)] * 6
        self.wrap = self.bc[4][0] == "periodic"
        self.device = torch.device("cuda", torch.cuda.current_device())
        stream = torch.cuda.current_stream().cuda_stream
        self.grid = Grid((self.shape[0], self.shape[1], self.z1 - self.z0), h=h, storage=storage, stream=stream)
        self.grid.set_bcs(slab_faces(self.bc, rank, world))
        self.kvar = False

    def close(self):
        self.grid.close()

    def _views(self, what):
        """(send_lo, send_hi, recv_lo, recv_hi) tensors over the slab's planes."""
        out = {}
        for face in (ZLO, ZHI):
            if self.grid_face_is_exchange(face):
                s, r, b = self.grid.exchange_planes(face, what)
                out[face] = (plane_tensor(s, b, self.device), plane_tensor(r, b, self.device))
            else:
                out[face] = (None, None)
        return out[ZLO][0], out[ZHI][0], out[ZLO][1], out[ZHI][1]

    def grid_face_is_exchange(self, face):
        return slab_faces(self.bc, self.rank, self.world)[face][0] == "exchange"

    def _exchange(self, what):
        s_lo, s_hi, r_lo, r_hi = self._views(what)
        exchange_halos(self.dist, self.rank, self.world, s_lo, s_hi, r_lo, r_hi, self.wrap)

    def set_field(self, T_slab):
        self.grid.set_field(T_slab)

    def set_coeffs(self, k_slab=1.0, u=(0.0, 0.0, 0.0)):
        self.grid.set_coeffs(k_slab, u)
        self.kvar = not np.isscalar(k_slab)
        if self.kvar:
            self._exchange(PLANES_K)
            self._exchange(PLANES_RECIP_K)

    def stability_dt(self):
        return allreduce_min(self.dist, self.grid.stability_dt(), self.device)

    def set_dt(self, dt):
        self.grid.set_dt(dt)

    def step(self, n):
        for _ in range(int(n)):
            self._exchange(PLANES_FIELD)
            self.grid.step(1)

    def total_heat(self):
        return allreduce_sum(self.dist, self.grid.total_heat(), self.device)
