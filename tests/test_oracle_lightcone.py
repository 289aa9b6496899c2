"""The oracle on a widened sub-box (oracle/lightcone.py) reproduces the
whole-grid oracle on the target box: after n steps a cell depends only on the
cells within n of it (Eq. expl_form couples face neighbours only), so the cut
faces of the widened box cannot reach the target. Checked against whole-grid
runs on small grids for every boundary kind, per-cell k and advection, and a
planted mistake (a box widened by n - 1) is caught."""
import numpy as np
import pytest

import oracle
from oracle import lightcone

D, ZF, P, DC = "dirichlet", "zeroflux", "periodic", "dirichlet_cell"

MIXES = [
    [(D, 1.0), (D, 0.0), (ZF, 0.0), (ZF, 0.0), (ZF, 0.0), (ZF, 0.0)],
    [(P, 0.0), (P, 0.0), (ZF, 0.0), (ZF, 0.0), (D, 0.3), (ZF, 0.0)],
    [(DC, 0.5), (D, -1.0), (P, 0.0), (P, 0.0), (ZF, 0.0), (DC, 0.2)],
    [(P, 0.0), (P, 0.0), (P, 0.0), (P, 0.0), (P, 0.0), (P, 0.0)],
]


def _problem(shape, seed, adv):
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    T0 = rng.uniform(0.0, 1.0, (nz, ny, nx))
    k = np.exp(0.5 * rng.standard_normal((nz, ny, nx)))
    u = (0.3, -0.2, 0.1) if adv else (0.0, 0.0, 0.0)
    return T0, k, u


@pytest.mark.parametrize("mix", range(len(MIXES)))
@pytest.mark.parametrize("adv", [False, True])
def test_box_equals_whole_grid(mix, adv):
    shape = (23, 19, 17)
    bc = MIXES[mix]
    T0, k, u = _problem(shape, 10 + mix, adv)
    dt = 0.9 * oracle.dt_max(shape=shape, k=k, u=u, bc=bc)
    n = 4
    whole = oracle.run(T0, n, shape=shape, k=k, u=u, bc=bc, dt=dt)
    boxes = [((0, 0, 0), (5, 4, 3)), ((18, 15, 14), (23, 19, 17)), ((8, 7, 6), (14, 12, 11)),
             ((20, 0, 5), (23, 19, 9)), ((0, 10, 0), (23, 12, 17))]
    for lo, hi in boxes:
        got = lightcone.run_box(T0, n, shape=shape, lo=lo, hi=hi, k=k, u=u, bc=bc, dt=dt)
        ref = whole[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14, err_msg=f"box {lo} {hi}")


def test_box_with_rounding_equals_whole_grid():
    shape = (21, 18, 16)
    bc = MIXES[1]
    T0, k, u = _problem(shape, 7, True)
    dt = 0.9 * oracle.dt_max(shape=shape, k=k, u=u, bc=bc)
    n = 5
    whole = oracle.run(oracle.round_to(T0, "bf16"), n, shape=shape, k=k, u=u, bc=bc, dt=dt, round_to="bf16")
    lo, hi = (15, 2, 3), (21, 9, 8)
    got = lightcone.run_box(T0, n, shape=shape, lo=lo, hi=hi, k=k, u=u, bc=bc, dt=dt, round_to="bf16")
    np.testing.assert_array_equal(got, whole[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]])


def test_too_narrow_a_box_is_caught():
    """A box widened by n - 1 instead of n lets a cut face reach the target:
    the comparison above would fail (so it can tell)."""
    shape = (23, 19, 17)
    bc = MIXES[0]
    T0, k, u = _problem(shape, 3, False)
    dt = 0.9 * oracle.dt_max(shape=shape, k=k, u=u, bc=bc)
    n = 4
    whole = oracle.run(T0, n, shape=shape, k=k, u=u, bc=bc, dt=dt)
    lo, hi = (8, 7, 6), (14, 12, 11)
    idx, faces, target = lightcone.cone_box(shape, bc, lo, hi, n - 1)
    sel = np.ix_(idx[2], idx[1], idx[0])
    R = oracle.run(T0[sel], n, shape=tuple(len(i) for i in idx), k=k[sel], bc=faces, dt=dt)
    bad = R[target[2], target[1], target[0]]
    assert np.abs(bad - whole[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]).max() > 1e-6


def test_target_outside_the_grid_is_rejected():
    with pytest.raises(ValueError):
        lightcone.cone_box((8, 8, 8), MIXES[0], (0, 0, 0), (9, 2, 2), 1)
