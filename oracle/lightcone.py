"""Oracle values on sub-boxes of a large grid (domain of dependence).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): used by the tests and
by the accuracy sample of ``bench.py``, never by the library.

The explicit step (Eq. expl_form) couples a cell to its six face neighbours
only, so after n steps a cell depends on the cells within n of it along each
axis (a box of radius n, the stencil's domain of dependence). To get the
oracle's field on a target box [lo, hi) of a grid too large to step whole,
this module cuts the target box widened by n on every side out of the full
inputs, runs ``oracle.run`` on it for n steps and returns the target part:

* a widened side that reaches a real boundary face keeps that face's
  condition (the box is clipped to the domain there);
* a side cut through the interior gets a zero-flux face: whatever it does,
  its influence moves one cell a step and cannot reach the target within n
  steps;
* a periodic axis whose widened box covers the whole period stays periodic;
  otherwise its indices wrap around the period and both cut faces are
  zero-flux.

The result on the target box equals the whole-grid oracle's there (the same
fp64 arithmetic on the same operands; ``tests/test_oracle_pins.py`` checks
that on small grids).
"""
from __future__ import annotations

import numpy as np

import oracle

ZF = ("zeroflux", 0.0)


def cone_box(shape, bc, lo, hi, n):
    """Index arrays, faces and target slice of the widened box.

    shape: (nx, ny, nz); bc: six (kind, value) pairs; lo, hi: target corner
    cells (x, y, z), hi exclusive; n: steps. Returns (idx, faces, target)
    where idx[a] are the grid indices along axis a (x, y, z), faces the six
    faces of the box and target[a] the slice of the target inside the box."""
    idx, faces, target = [], [], []
    for a in range(3):
        N = shape[a]
        l, h = int(lo[a]), int(hi[a])
        if not 0 <= l < h <= N:
            raise ValueError(f"target box [{l}, {h}) outside axis {a} of length {N}")
        lo_kind, hi_kind = bc[2 * a], bc[2 * a + 1]
        periodic = lo_kind[0] == "periodic"
        if periodic and (h - l) + 2 * n >= N:
            ix = np.arange(N)
            faces += [lo_kind, hi_kind]
            target.append(slice(l, h))
        elif periodic:
            ix = np.arange(l - n, h + n) % N
            faces += [ZF, ZF]
            target.append(slice(n, n + h - l))
        else:
            a0, a1 = max(0, l - n), min(N, h + n)
            ix = np.arange(a0, a1)
            faces += [lo_kind if a0 == 0 else ZF, hi_kind if a1 == N else ZF]
            target.append(slice(l - a0, h - a0))
        idx.append(ix)
    return idx, faces, target


def run_box(T0, n, *, shape, lo, hi, h=(1.0, 1.0, 1.0), k=1.0, u=(0.0, 0.0, 0.0), bc, dt, round_to=None,
            threads=0):
    """The oracle's field after n steps on the target box [lo, hi) (x, y, z
    corners, hi exclusive) of the grid `shape`, as an array indexed [z, y, x].
    T0 and an array k are the full grid's inputs ([z, y, x]); round_to as in
    ``oracle.run`` (the initial field is rounded the same way first)."""
    idx, faces, target = cone_box(shape, bc, lo, hi, n)
    sel = np.ix_(idx[2], idx[1], idx[0])
    T = np.asarray(T0[sel], dtype=np.float64)
    if round_to:
        T = oracle.round_to(T, round_to).astype(np.float64)
    kk = k if np.isscalar(k) else np.asarray(k[sel], dtype=np.float64)
    box = (len(idx[0]), len(idx[1]), len(idx[2]))
    R = oracle.run(T, n, shape=box, h=h, k=kk, u=u, bc=faces, dt=dt, round_to=round_to, threads=threads)
    return R[target[2], target[1], target[0]]
