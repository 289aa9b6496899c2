"""Pins for the oracle's implicit step (backward Euler solved by classic CG,
Sec. 1.1.2, Eq. impl_form), CPU only.

The CG result is checked against a dense LAPACK solve of the system assembled
cell by cell from the explicit stepping matrix (itself pinned in
test_oracle_pins), whole-field solutions in the DST / DCT / FFT eigenbasis
for uniform k, the paper's own form of the equation with held boundary
cells, conservation, the maximum principle, and two properties of CG itself:
a single eigenmode converges in one iteration, and a system with m distinct
eigenvalues in at most m.
"""
import os

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
from test_oracle_pins import BC_MIXES, D, DC, P, ZF, _apply_held, _bc, _mode_1d, _spectral_solution, brute_matrix


def dense_implicit(T0, steps, shape, h, k, bc, dt):
    """Backward Euler by dense solves: with the explicit step T' = M T + b,
    M = I + dt L on free rows, the implicit step solves (2 I - M) T' = T + b
    on free rows and T' = value on held rows."""
    M, b, held = brute_matrix(shape, h, k, (0.0, 0.0, 0.0), bc, dt)
    N = M.shape[0]
    A = 2.0 * np.eye(N) - M
    T = np.asarray(T0, dtype=np.float64).ravel().copy()
    for C, val in held.items():
        A[C, :] = 0.0
        A[C, C] = 1.0
    for _ in range(steps):
        rhs = T + b
        for C, val in held.items():
            rhs[C] = val
        T = np.linalg.solve(A, rhs)
    return T.reshape(np.shape(T0)), A, held


@pytest.mark.parametrize("mix", range(len(BC_MIXES)))
@pytest.mark.parametrize("kvar", [False, True])
def test_implicit_matches_dense_solve(mix, kvar):
    rng = np.random.default_rng(200 + mix)
    shape = (5, 4, 6)
    nx, ny, nz = shape
    h = (1.1, 0.8, 1.3)
    k = np.exp(0.5 * rng.standard_normal((nz, ny, nx))) if kvar else 0.9
    bc = _bc(BC_MIXES[mix], list(rng.uniform(-1, 2, 6)))
    dt = 0.7   # far above the explicit limit: backward Euler is stable at any dt
    T0 = rng.uniform(0, 1, (nz, ny, nx))
    ref, _, held = dense_implicit(T0, 2, shape, h, k, bc, dt)
    T, iters, res = oracle.implicit(T0, 2, shape=shape, h=h, k=k, bc=bc, dt=dt, rtol=1e-14)
    assert res <= 1e-14 and iters > 0
    np.testing.assert_allclose(T, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("kinds", [(D, D, D), (ZF, D, ZF), (P, P, P), (P, ZF, D), (DC, DC, DC), (DC, P, ZF)])
def test_implicit_spectral_whole_field(kinds):
    rng = np.random.default_rng(12)
    shape = (10, 9, 7)
    h = (1.0, 0.9, 1.2)
    kval = 0.6
    bc = _bc([kinds[0]] * 2 + [kinds[1]] * 2 + [kinds[2]] * 2)
    T0 = rng.uniform(0, 1, shape[::-1])
    for a in range(3):   # held layers carry 0 (the value of every face here)
        if kinds[a] == DC:
            idx = [slice(None)] * 3
            idx[2 - a] = 0
            T0[tuple(idx)] = 0
            idx[2 - a] = -1
            T0[tuple(idx)] = 0
    dt = 2.5
    T, _, _ = oracle.implicit(T0, 3, shape=shape, h=h, k=kval, bc=bc, dt=dt, rtol=1e-14)
    ref = _spectral_solution(T0, 3, shape, h, kval, (0, 0, 0), kinds, dt, implicit=True)
    np.testing.assert_allclose(T, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("kinds,modes", [((D, D, D), (1, 2, 3)), ((ZF, ZF, ZF), (1, 0, 2)), ((P, P, P), (1, 2, 1)),
                                         ((DC, DC, DC), (1, 1, 2)), ((D, ZF, P), (2, 3, 1))])
def test_implicit_single_mode_one_iteration(kinds, modes):
    # r0 = b - A T^n = -dt rate T^n is an eigenvector of A: CG is exact after
    # one iteration, and the mode is divided by 1 + dt rate per step
    shape = (12, 10, 8)
    h = (1.0, 0.8, 1.3)
    kval = 0.7
    bc = _bc([kinds[0]] * 2 + [kinds[1]] * 2 + [kinds[2]] * 2)
    vecs, lam = [], 0.0
    for a in range(3):
        v, ev = _mode_1d(kinds[a], shape[a], modes[a])
        vecs.append(v)
        lam += kval * ev / h[a] ** 2
    T0 = np.einsum("z,y,x->zyx", vecs[2], vecs[1], vecs[0])
    dt, n = 0.8, 4
    T, iters, res = oracle.implicit(T0, n, shape=shape, h=h, k=kval, bc=bc, dt=dt, rtol=1e-12)
    assert iters == n and res <= 1e-12
    np.testing.assert_allclose(T, T0 / (1.0 + dt * lam) ** n, rtol=0, atol=1e-13)


def test_implicit_iterations_bounded_by_distinct_eigenvalues():
    # in exact arithmetic CG ends after at most as many iterations as A has
    # distinct eigenvalues; a uniform-k box with held x layers has few
    shape = (5, 4, 4)
    bc = _bc([DC, DC, P, P, P, P])
    T0 = np.random.default_rng(4).uniform(0, 1, shape[::-1])
    _, A, held = dense_implicit(T0, 1, shape, (1.0, 1.0, 1.0), 1.0, bc, 0.9)
    free = [c for c in range(A.shape[0]) if c not in held]
    ev = np.linalg.eigvalsh(A[np.ix_(free, free)])
    distinct = len(np.unique(np.round(ev, 9)))
    assert distinct < len(free)
    _, iters, res = oracle.implicit(T0, 1, shape=shape, k=1.0, bc=bc, dt=0.9, rtol=1e-12)
    assert iters <= distinct and res <= 1e-12


def test_implicit_cg_error_decreases_in_energy_norm():
    # the k-th CG iterate minimises the A-norm of the error over the Krylov
    # space, so the error never grows from one iteration to the next
    rng = np.random.default_rng(8)
    shape = (6, 5, 4)
    nx, ny, nz = shape
    k = np.exp(0.5 * rng.standard_normal((nz, ny, nx)))
    bc = _bc([D, ZF, ZF, ZF, P, P], list(rng.uniform(0, 1, 6)))
    T0 = rng.uniform(0, 1, (nz, ny, nx))
    ref, A, held = dense_implicit(T0, 1, shape, (1.0, 1.0, 1.0), k, bc, 1.5)
    prev = np.inf
    for m in list(range(0, 12)) + [20, 40, 80]:
        T, iters, _ = oracle.implicit(T0, 1, shape=shape, k=k, bc=bc, dt=1.5, rtol=0.0, max_iter=m)
        assert iters == m
        e = (T - ref).ravel()
        err = float(e @ (A @ e))
        assert err <= prev * (1 + 1e-12)
        prev = err
    assert prev < 1e-20


def test_implicit_paper_form_held_cells():
    # uniform k = 1, h = 1, held layers on every face: Eq. impl_form verbatim,
    # T'_C - omega psi sum_D T'_D = psi T_C, psi = 1 / (1 + 6 omega)
    rng = np.random.default_rng(31)
    shape = (9, 8, 7)
    gam = list(rng.uniform(0, 1, 6))
    bc = _bc([DC] * 6, gam)
    omega = 0.1
    T0 = oracle.run(rng.uniform(0, 1, shape[::-1]), 0, shape=shape, k=1.0, bc=bc, dt=omega)
    T1, _, _ = oracle.implicit(T0, 1, shape=shape, k=1.0, bc=bc, dt=omega, rtol=1e-14)
    psi = 1.0 / (1.0 + 6.0 * omega)
    w = np.zeros((3, 3, 3))
    w[1, 1, 0] = w[1, 1, 2] = w[1, 0, 1] = w[1, 2, 1] = w[0, 1, 1] = w[2, 1, 1] = 1.0
    nb = ndi.correlate(T1, w, mode="constant")
    lhs = T1 - omega * psi * nb
    np.testing.assert_allclose(lhs[1:-1, 1:-1, 1:-1], psi * T0[1:-1, 1:-1, 1:-1], rtol=0, atol=1e-13)
    np.testing.assert_array_equal(T1[:, :, 0], T0[:, :, 0])
    np.testing.assert_array_equal(T1[-1], T0[-1])


@pytest.mark.parametrize("kinds", [(ZF, ZF, ZF), (P, ZF, P), (P, P, P)])
def test_implicit_conservation(kinds):
    rng = np.random.default_rng(15)
    shape = (14, 11, 9)
    k = np.exp(0.5 * rng.standard_normal(shape[::-1]))
    bc = _bc([kinds[0]] * 2 + [kinds[1]] * 2 + [kinds[2]] * 2)
    T0 = rng.uniform(0, 1, shape[::-1])
    T, _, _ = oracle.implicit(T0, 5, shape=shape, k=k, bc=bc, dt=3.0, rtol=1e-14)
    assert abs(T.sum() - T0.sum()) <= 1e-11 * T0.sum()


def test_implicit_maximum_principle():
    # A is an M-matrix: the solution stays within the range of T^n and of the
    # boundary values
    rng = np.random.default_rng(16)
    shape = (13, 10, 8)
    k = np.exp(0.8 * rng.standard_normal(shape[::-1]))
    bc = _bc([D, DC, ZF, D, P, P], [0.1, 0.9, 0.0, 0.3, 0.0, 0.0])
    T0 = rng.uniform(0.1, 0.9, shape[::-1])
    T, _, _ = oracle.implicit(T0, 4, shape=shape, k=k, bc=bc, dt=10.0, rtol=1e-13)
    assert T.min() >= 0.1 - 1e-12 and T.max() <= 0.9 + 1e-12


def test_implicit_zero_steps_and_rejects():
    T0 = np.random.default_rng(1).uniform(0, 1, (3, 4, 5))
    bc = _bc([DC, D, ZF, ZF, P, P], [0.5, 0, 0, 0, 0, 0])
    T, iters, _ = oracle.implicit(T0, 0, shape=(5, 4, 3), k=1.0, bc=bc, dt=1.0)
    assert iters == 0
    np.testing.assert_array_equal(T[:, :, 1:], T0[:, :, 1:])
    assert (T[:, :, 0] == 0.5).all()   # held layers take their value
    with pytest.raises(ValueError):
        oracle.implicit(T0, 1, shape=(5, 4, 3), k=1.0, bc=_bc([P, D, ZF, ZF, P, P]), dt=1.0)
    with pytest.raises(ValueError):
        oracle.implicit(T0, 1, shape=(5, 4, 3), k=1.0, bc=bc, dt=-1.0)


@pytest.mark.parametrize("mix", [0, 3, 4, 5, 6])
def test_cgcg_iterates_equal_classic_cg(mix):
    # Chronopoulos-Gear CG carries A r and A p by recurrence; in exact
    # arithmetic its iterates are classic CG's, so every fixed iteration count
    # must agree to rounding
    rng = np.random.default_rng(300 + mix)
    shape = (7, 5, 6)
    nx, ny, nz = shape
    k = np.exp(0.5 * rng.standard_normal((nz, ny, nx)))
    bc = _bc(BC_MIXES[mix], list(rng.uniform(-1, 2, 6)))
    T0 = rng.uniform(0, 1, (nz, ny, nx))
    for m in (1, 2, 4, 8, 15):
        a, ia, _ = oracle.implicit(T0, 1, shape=shape, k=k, bc=bc, dt=2.0, rtol=0.0, max_iter=m)
        b, ib, _ = oracle.implicit(T0, 1, shape=shape, k=k, bc=bc, dt=2.0, rtol=0.0, max_iter=m, method="cgcg")
        assert ia == ib == m
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-12)


@pytest.mark.parametrize("mix", [1, 2, 4])
def test_cgcg_matches_dense_solve(mix):
    rng = np.random.default_rng(310 + mix)
    shape = (5, 4, 6)
    nx, ny, nz = shape
    k = np.exp(0.5 * rng.standard_normal((nz, ny, nx)))
    bc = _bc(BC_MIXES[mix], list(rng.uniform(-1, 2, 6)))
    T0 = rng.uniform(0, 1, (nz, ny, nx))
    ref, _, _ = dense_implicit(T0, 2, shape, (1.1, 0.8, 1.3), k, bc, 0.7)
    T, _, res = oracle.implicit(T0, 2, shape=shape, h=(1.1, 0.8, 1.3), k=k, bc=bc, dt=0.7, rtol=1e-14,
                                method="cgcg")
    assert res <= 1e-14
    np.testing.assert_allclose(T, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("method", ["classic", "cgcg"])
def test_implicit_thread_count_does_not_change_results(method):
    # the face passes run in parallel over lines (no shared accumulator) and
    # the inner products are sequential: any thread count, the same bits
    rng = np.random.default_rng(17)
    shape = (23, 17, 11)
    k = np.exp(0.5 * rng.standard_normal(shape[::-1]))
    bc = _bc(BC_MIXES[4], list(rng.uniform(0, 1, 6)))
    T0 = rng.uniform(0, 1, shape[::-1])
    a = oracle.implicit(T0, 2, shape=shape, k=k, bc=bc, dt=1.5, rtol=1e-10, threads=1, method=method)
    b = oracle.implicit(T0, 2, shape=shape, k=k, bc=bc, dt=1.5, rtol=1e-10, threads=4, method=method)
    oracle.implicit(T0, 0, shape=shape, k=k, bc=bc, dt=1.5, threads=os.cpu_count() or 1)   # restore
    assert a[1] == b[1]
    np.testing.assert_array_equal(a[0], b[0])
