"""Pins for the FP64 oracle (CPU only).

Each test checks the oracle against something other than its own code:
hand-derived values (tests/golden), closed-form eigen-decays, whole-field
solutions through scipy's DST/DCT/FFT (the discrete operator is diagonal in
those bases for uniform k), invariants (conservation, maximum principle, a
layered steady state) and a dense-matrix stepper assembled cell by cell from a
separate "ghost value" formulation. Together they catch a dropped term, a
wrong sign or index, or a transposed operand anywhere in the oracle.
"""
import os

import numpy as np
import pytest
import scipy.fft as sfft
import scipy.ndimage as ndi

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

D, ZF, P, DC = "dirichlet", "zeroflux", "periodic", "dirichlet_cell"


def _bc(kinds, values=None):
    values = values or [0.0] * 6
    return [(k, v) for k, v in zip(kinds, values)]


# --------------------------------------------------------------------------
# dense-matrix stepper: T' = M T + b, assembled per cell (gather form)
# --------------------------------------------------------------------------
def brute_matrix(shape, h, k, u, bc, dt):
    nx, ny, nz = shape
    N = nx * ny * nz
    kk = np.broadcast_to(np.asarray(k, dtype=np.float64), (nz, ny, nx)).ravel()
    M = np.zeros((N, N))
    b = np.zeros(N)

    def index(c):
        return c[0] + nx * (c[1] + ny * c[2])

    held = {}
    for f, (kind, val) in enumerate(bc):
        if kind != DC:
            continue
        a = f // 2
        want = 0 if f % 2 == 0 else shape[a] - 1
        for l in range(nz):
            for j in range(ny):
                for i in range(nx):
                    if (i, j, l)[a] == want:
                        held[index((i, j, l))] = val
    for l in range(nz):
        for j in range(ny):
            for i in range(nx):
                C = index((i, j, l))
                if C in held:
                    b[C] = held[C]
                    continue
                M[C, C] = 1.0
                kC = kk[C]
                for a in range(3):
                    ha = h[a]
                    up, um = max(u[a], 0.0), min(u[a], 0.0)
                    for side in (-1, 1):
                        f = 2 * a + (0 if side < 0 else 1)
                        kind, val = bc[f]
                        c = [i, j, l]
                        c[a] += side
                        inside = 0 <= c[a] < shape[a]
                        if not inside and kind == P:
                            c[a] %= shape[a]
                            inside = True
                        if inside:
                            Dn = index(c)
                            kD = kk[Dn]
                            K = 2 * kC * kD / (kC + kD) if kC + kD > 0 else 0.0
                            M[C, Dn] += dt * K / ha**2
                            M[C, C] -= dt * K / ha**2
                            if side < 0:   # flux u+ T_W + u- T_C enters through the low face
                                M[C, Dn] += dt * up / ha
                                M[C, C] += dt * um / ha
                            else:          # flux u+ T_C + u- T_E leaves through the high face
                                M[C, C] -= dt * up / ha
                                M[C, Dn] -= dt * um / ha
                        elif kind == D:
                            M[C, C] -= dt * 2 * kC / ha**2
                            b[C] += dt * 2 * kC / ha**2 * val
                            if side < 0:
                                b[C] += dt * up / ha * val
                                M[C, C] += dt * um / ha
                            else:
                                M[C, C] -= dt * up / ha
                                b[C] -= dt * um / ha * val
    return M, b, held


def _apply_held(T, shape, held):
    t = T.ravel().copy()
    for c, v in held.items():
        t[c] = v
    return t.reshape(T.shape)


# --------------------------------------------------------------------------
# hand values (Eq. expl_form, omega = 1/10)
# --------------------------------------------------------------------------
def _golden():
    cases = {}
    with open(os.path.join(GOLDEN, "hand_4x4x4.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, x, y, z, v = line.split()
            cases.setdefault(name, []).append((int(x), int(y), int(z), float(v)))
    return cases


def test_hand_values_4x4x4():
    cases = _golden()
    bc = _bc([D] * 6)
    for name, pulse in (("interior", (1, 1, 1)), ("corner", (0, 0, 0))):
        T0 = np.zeros((4, 4, 4))
        T0[pulse[2], pulse[1], pulse[0]] = 1.0
        T1 = oracle.run(T0, 1, shape=(4, 4, 4), k=1.0, bc=bc, dt=0.1)
        expect = np.zeros_like(T1)
        for x, y, z, v in cases[name]:
            expect[z, y, x] = v
        np.testing.assert_allclose(T1, expect, rtol=0, atol=1e-15)
    assert abs(oracle.total_heat(T1) - 0.4) < 1e-15
    # harmonic-mean face conductivity k = (1, 3) -> 1.5
    T0 = np.array([[[1.0, 0.0]]])
    k = np.array([[[1.0, 3.0]]])
    T1 = oracle.run(T0, 1, shape=(2, 1, 1), k=k, bc=_bc([ZF] * 6), dt=0.1)
    for x, y, z, v in cases["harmonic"]:
        assert abs(T1[z, y, x] - v) < 1e-15


def test_dt_limit_matches_paper_omega():
    # face Dirichlet on all faces, k = h = 1: corner cells couple 3*1 + 3*2 = 9,
    # so 0.9 * dt_max = 0.1 = the omega of Sec. 1.1.1
    assert abs(oracle.dt_max(shape=(64, 64, 64), k=1.0, bc=_bc([D] * 6)) - 1 / 9) < 1e-16
    # held boundary cells (Eq. expl_form verbatim): interior cells couple 6 -> 1/6
    assert abs(oracle.dt_max(shape=(8, 8, 8), k=1.0, bc=_bc([DC] * 6)) - 1 / 6) < 1e-16
    # no coupling at all
    assert oracle.dt_max(shape=(4, 4, 4), k=0.0, bc=_bc([ZF] * 6)) == np.inf


# --------------------------------------------------------------------------
# dense-matrix equality over random problems and every boundary mix
# --------------------------------------------------------------------------
BC_MIXES = [
    [D, D, D, D, D, D],
    [ZF, ZF, ZF, ZF, ZF, ZF],
    [P, P, P, P, P, P],
    [DC, DC, DC, DC, DC, DC],
    [D, ZF, P, P, DC, D],
    [DC, D, ZF, DC, P, P],
    [P, P, D, ZF, ZF, D],
]


@pytest.mark.parametrize("mix", range(len(BC_MIXES)))
@pytest.mark.parametrize("shape", [(4, 3, 5), (2, 6, 3), (5, 5, 2)])
def test_brute_force_matrix(mix, shape):
    rng = np.random.default_rng(100 + mix)
    nx, ny, nz = shape
    k = np.exp(0.5 * rng.standard_normal((nz, ny, nx)))
    u = tuple(rng.uniform(-0.4, 0.4, 3))
    h = tuple(rng.uniform(0.7, 1.5, 3))
    bc = _bc(BC_MIXES[mix], list(rng.uniform(-1, 2, 6)))
    dtm = oracle.dt_max(shape=shape, h=h, k=k, u=u, bc=bc)
    dt = 0.9 * dtm
    M, b, held = brute_matrix(shape, h, k, u, bc, dt)
    T0 = _apply_held(rng.uniform(0, 1, (nz, ny, nx)), shape, held)
    T_brute = T0.ravel()
    for _ in range(5):
        T_brute = M @ T_brute + b
    T_or = oracle.run(T0, 5, shape=shape, h=h, k=k, u=u, bc=bc, dt=dt)
    scale = max(1.0, np.abs(T_brute).max())
    np.testing.assert_allclose(T_or.ravel(), T_brute, rtol=0, atol=1e-13 * scale)
    if not np.isfinite(dtm):   # every cell is held: nothing to limit
        assert len(held) == nx * ny * nz
        return
    # the positivity limit: every weight of M is >= 0 at dt_max and not above it
    M1, _, _ = brute_matrix(shape, h, k, u, bc, dtm)
    assert M1.min() >= -1e-13
    M2, _, _ = brute_matrix(shape, h, k, u, bc, 1.02 * dtm)
    assert M2.min() < -1e-6


def test_held_layer_priority():
    # a cell on two held layers takes the value of the later face (-x,+x,-y,+y,-z,+z)
    shape = (4, 4, 4)
    bc = _bc([DC, ZF, DC, ZF, ZF, ZF], [1.0, 0, 2.0, 0, 0, 0])
    T = oracle.run(np.zeros((4, 4, 4)), 1, shape=shape, k=1.0, bc=bc, dt=0.1)
    assert T[0, 0, 0] == 2.0 and T[0, 1, 0] == 1.0 and T[0, 0, 1] == 2.0
    M, b, held = brute_matrix(shape, (1, 1, 1), 1.0, (0, 0, 0), bc, 0.1)
    assert held[0] == 2.0


# --------------------------------------------------------------------------
# closed-form eigen-decay of single modes (uniform k)
# --------------------------------------------------------------------------
def _mode_1d(kind, n, m):
    i = np.arange(n, dtype=np.float64)
    if kind == D:      # sin(pi m (i + 1/2) / N), eigenvalue 4 sin^2(pi m / 2N)
        return np.sin(np.pi * m * (i + 0.5) / n), 4 * np.sin(np.pi * m / (2 * n)) ** 2
    if kind == ZF:     # cos(pi m (i + 1/2) / N)
        return np.cos(np.pi * m * (i + 0.5) / n), 4 * np.sin(np.pi * m / (2 * n)) ** 2
    if kind == P:      # cos(2 pi m i / N), eigenvalue 4 sin^2(pi m / N)
        return np.cos(2 * np.pi * m * i / n), 4 * np.sin(np.pi * m / n) ** 2
    if kind == DC:     # sin(pi m i / (N - 1)): zero on the held layers
        return np.sin(np.pi * m * i / (n - 1)), 4 * np.sin(np.pi * m / (2 * (n - 1))) ** 2
    raise ValueError(kind)


@pytest.mark.parametrize("kinds,modes", [
    ((D, D, D), (1, 2, 3)),
    ((ZF, ZF, ZF), (1, 0, 2)),
    ((P, P, P), (1, 2, 1)),
    ((DC, DC, DC), (1, 1, 2)),
    ((D, ZF, P), (2, 3, 1)),
])
def test_single_mode_decay(kinds, modes):
    shape = (12, 10, 8)
    h = (1.0, 0.8, 1.3)
    kval = 0.7
    bc = _bc([kinds[0]] * 2 + [kinds[1]] * 2 + [kinds[2]] * 2)
    dt = 0.9 * oracle.dt_max(shape=shape, h=h, k=kval, bc=bc)
    vecs, lam = [], 0.0
    for a in range(3):
        v, ev = _mode_1d(kinds[a], shape[a], modes[a])
        vecs.append(v)
        lam += kval * ev / h[a] ** 2
    T0 = np.einsum("z,y,x->zyx", vecs[2], vecs[1], vecs[0])
    g = 1.0 - dt * lam
    n = 40
    T = oracle.run(T0, n, shape=shape, h=h, k=kval, bc=bc, dt=dt)
    np.testing.assert_allclose(T, g**n * T0, rtol=0, atol=1e-13)


def test_advection_fourier_mode():
    shape = (16, 12, 10)
    h = (1.0, 1.0, 1.0)
    u = (0.3, -0.1, 0.05)
    kval = 0.05
    bc = _bc([P] * 6)
    dt = 1.0
    m = (2, 1, 3)
    theta = [2 * np.pi * m[a] / shape[a] for a in range(3)]
    g = 1.0 + 0j
    for a in range(3):
        cp, cm = dt * max(u[a], 0) / h[a], dt * max(-u[a], 0) / h[a]
        d = kval * dt / h[a] ** 2
        g += cp * (np.exp(-1j * theta[a]) - 1) + cm * (np.exp(1j * theta[a]) - 1) \
            + d * (2 * np.cos(theta[a]) - 2)
    z, y, x = np.meshgrid(*(np.arange(s) for s in shape[::-1]), indexing="ij")
    phase = np.exp(1j * (theta[0] * x + theta[1] * y + theta[2] * z))
    A = 0.8 * np.exp(0.3j)
    T0 = np.real(A * phase)
    n = 25
    T = oracle.run(T0, n, shape=shape, h=h, k=kval, u=u, bc=bc, dt=dt)
    np.testing.assert_allclose(T, np.real(A * g**n * phase), rtol=0, atol=1e-13)


def test_integer_shift_courant_one():
    # pure upwind advection at Courant number 1 moves the field exactly one cell
    rng = np.random.default_rng(7)
    shape = (9, 5, 4)
    T0 = rng.integers(-50, 50, (4, 5, 9)).astype(np.float64)
    bc = _bc([P] * 6)
    T = oracle.run(T0, 3, shape=shape, k=0.0, u=(1.0, 0.0, 0.0), bc=bc, dt=1.0)
    np.testing.assert_array_equal(T, np.roll(T0, 3, axis=2))
    T = oracle.run(T0, 2, shape=shape, k=0.0, u=(0.0, 0.0, -1.0), bc=bc, dt=1.0)
    np.testing.assert_array_equal(T, np.roll(T0, -2, axis=0))


# --------------------------------------------------------------------------
# whole-field solutions through scipy transforms (uniform k, random field)
# --------------------------------------------------------------------------
def _spectral_solution(T0, n, shape, h, kval, u, kinds, dt, implicit=False):
    """n steps of the uniform-k operator, axis by axis in its eigenbasis
    (explicit: each mode times 1 - dt rate; implicit, backward Euler: divided
    by 1 + dt rate)."""
    X = np.asarray(T0, dtype=np.float64)
    sl = [slice(None)] * 3
    # forward transforms, axis 2 of the array is x
    plan = []
    for a in range(3):
        ax = 2 - a
        kind = kinds[a]
        N = shape[a]
        if kind == D:
            X = sfft.dst(X, type=2, axis=ax, norm="ortho")
            m = np.arange(1, N + 1)
            lam = 4 * np.sin(np.pi * m / (2 * N)) ** 2
            adv = np.zeros(N)
        elif kind == ZF:
            X = sfft.dct(X, type=2, axis=ax, norm="ortho")
            m = np.arange(N)
            lam = 4 * np.sin(np.pi * m / (2 * N)) ** 2
            adv = np.zeros(N)
        elif kind == P:
            X = sfft.fft(X, axis=ax)
            th = 2 * np.pi * np.fft.fftfreq(N)
            lam = 4 * np.sin(th / 2) ** 2 + 0j
            cp, cm = max(u[a], 0) / h[a], max(-u[a], 0) / h[a]
            adv = cp * (1 - np.exp(-1j * th)) + cm * (1 - np.exp(1j * th))
        elif kind == DC:
            inner = [slice(None)] * 3
            inner[ax] = slice(1, N - 1)
            X = X[tuple(inner)]
            X = sfft.dst(X, type=1, axis=ax, norm="ortho")
            m = np.arange(1, N - 1)
            lam = 4 * np.sin(np.pi * m / (2 * (N - 1))) ** 2
            adv = np.zeros(N - 2)
        plan.append((ax, kind, N))
        shp = [1, 1, 1]
        shp[ax] = -1
        rate = kval * lam / h[a] ** 2 + adv
        if a == 0:
            total = rate.reshape(shp)
        else:
            total = total + rate.reshape(shp)
    X = X * ((1.0 / (1.0 + dt * total)) if implicit else (1.0 - dt * total)) ** n
    for ax, kind, N in reversed(plan):
        if kind == D:
            X = sfft.idst(X, type=2, axis=ax, norm="ortho")
        elif kind == ZF:
            X = sfft.idct(X, type=2, axis=ax, norm="ortho")
        elif kind == P:
            X = sfft.ifft(X, axis=ax)
        elif kind == DC:
            X = sfft.idst(X, type=1, axis=ax, norm="ortho")
            pad = [(0, 0)] * 3
            pad[ax] = (1, 1)
            X = np.pad(X, pad)
    return np.real(X)


@pytest.mark.parametrize("kinds,u", [
    ((D, D, D), (0, 0, 0)),
    ((ZF, D, ZF), (0, 0, 0)),
    ((P, P, P), (0.3, -0.2, 0.1)),
    ((P, ZF, D), (0.4, 0, 0)),
    ((DC, DC, DC), (0, 0, 0)),
    ((DC, P, ZF), (0, -0.25, 0)),
])
def test_spectral_whole_field(kinds, u):
    rng = np.random.default_rng(11)
    shape = (10, 9, 7)
    h = (1.0, 0.9, 1.2)
    kval = 0.6
    bc = _bc([kinds[0]] * 2 + [kinds[1]] * 2 + [kinds[2]] * 2)
    dt = 0.9 * oracle.dt_max(shape=shape, h=h, k=kval, u=u, bc=bc)
    T0 = rng.uniform(0, 1, shape[::-1])
    for a in range(3):   # held layers carry 0 (the value of every face here)
        if kinds[a] == DC:
            idx = [slice(None)] * 3
            idx[2 - a] = 0
            T0[tuple(idx)] = 0
            idx[2 - a] = -1
            T0[tuple(idx)] = 0
    n = 30
    T = oracle.run(T0, n, shape=shape, h=h, k=kval, u=u, bc=bc, dt=dt)
    ref = _spectral_solution(T0, n, shape, h, kval, u, kinds, dt)
    np.testing.assert_allclose(T, ref, rtol=0, atol=1e-12)


def test_paper_form_held_cells():
    # uniform k with held boundary cells is Eq. expl_form verbatim:
    # T' = omega * sum of the 6 neighbours + (1 - 6 omega) T for interior cells
    rng = np.random.default_rng(3)
    shape = (9, 8, 7)
    gam = list(rng.uniform(0, 1, 6))
    bc = _bc([DC] * 6, gam)
    omega = 0.1
    T0 = rng.uniform(0, 1, shape[::-1])
    T1 = oracle.run(T0, 1, shape=shape, k=1.0, bc=bc, dt=omega)
    Tin = oracle.run(T0, 0, shape=shape, k=1.0, bc=bc, dt=omega)   # held layers applied
    w = np.zeros((3, 3, 3))
    w[1, 1, 0] = w[1, 1, 2] = w[1, 0, 1] = w[1, 2, 1] = w[0, 1, 1] = w[2, 1, 1] = omega
    w[1, 1, 1] = 1 - 6 * omega
    ref = ndi.correlate(Tin, w, mode="constant")
    np.testing.assert_allclose(T1[1:-1, 1:-1, 1:-1], ref[1:-1, 1:-1, 1:-1], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(T1[:, :, 0], Tin[:, :, 0])


# --------------------------------------------------------------------------
# invariants with variable k and advection
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kinds", [(ZF, ZF, ZF), (P, ZF, P), (P, P, P)])
def test_conservation(kinds):
    rng = np.random.default_rng(5)
    shape = (14, 11, 9)
    k = np.exp(0.5 * rng.standard_normal(shape[::-1]))
    u = (0.3, -0.1, 0.05)
    bc = _bc([kinds[0]] * 2 + [kinds[1]] * 2 + [kinds[2]] * 2)
    dt = 0.9 * oracle.dt_max(shape=shape, k=k, u=u, bc=bc)
    T0 = rng.uniform(0, 1, shape[::-1])
    E0 = oracle.total_heat(T0)
    T = oracle.run(T0, 60, shape=shape, k=k, u=u, bc=bc, dt=dt)
    assert abs(oracle.total_heat(T) - E0) <= 1e-12 * E0
    np.testing.assert_allclose(oracle.total_heat(T), T.sum(), rtol=1e-14)


def test_dirichlet_energy_balance():
    # E_{n+1} - E_n = dt * (net flux through the Dirichlet faces)
    rng = np.random.default_rng(6)
    shape = (6, 5, 4)
    h = (1.0, 0.5, 2.0)
    k = np.exp(0.5 * rng.standard_normal(shape[::-1]))
    bc = _bc([D, D, ZF, D, ZF, ZF], [1.0, -0.5, 0, 2.0, 0, 0])
    dt = 0.5 * oracle.dt_max(shape=shape, h=h, k=k, bc=bc)
    T0 = rng.uniform(0, 1, shape[::-1])
    T1 = oracle.run(T0, 1, shape=shape, h=h, k=k, bc=bc, dt=dt)
    vol = h[0] * h[1] * h[2]
    flux = 0.0
    # -x face (x = 0), +x face (x = nx - 1), +y face (y = ny - 1); area / distance
    flux += np.sum(2 * k[:, :, 0] * (1.0 - T0[:, :, 0])) * h[1] * h[2] / h[0]
    flux += np.sum(2 * k[:, :, -1] * (-0.5 - T0[:, :, -1])) * h[1] * h[2] / h[0]
    flux += np.sum(2 * k[:, -1, :] * (2.0 - T0[:, -1, :])) * h[0] * h[2] / h[1]
    dE = oracle.total_heat(T1, h) - oracle.total_heat(T0, h)
    assert abs(dE - dt * flux) < 1e-13 * max(1.0, abs(flux)) * vol



def test_dirichlet_energy_balance_with_advection():
    # with upwind advection: the net flux through a Dirichlet face carries T_b
    # where the flow enters and T_C where it leaves; zero-flux faces carry
    # nothing (the interior and periodic fluxes cancel in the sum)
    rng = np.random.default_rng(16)
    shape = (7, 5, 6)
    h = (1.0, 0.8, 1.3)
    u = (0.25, -0.2, 0.1)
    k = np.exp(0.5 * rng.standard_normal(shape[::-1]))
    bc = _bc([D, D, D, ZF, P, P], [0.7, -0.3, 1.5, 0, 0, 0])
    dt = 0.5 * oracle.dt_max(shape=shape, h=h, k=k, u=u, bc=bc)
    T0 = rng.uniform(0, 1, shape[::-1])
    T1 = oracle.run(T0, 1, shape=shape, h=h, k=k, u=u, bc=bc, dt=dt)
    ax, ay, az = h[1] * h[2], h[0] * h[2], h[0] * h[1]   # face areas
    flux = 0.0
    # -x (value 0.7): diffusion and inflow (u_x > 0 enters here with T_b)
    flux += np.sum(2 * k[:, :, 0] * (0.7 - T0[:, :, 0])) * ax / h[0] + u[0] * 0.7 * T0[:, :, 0].size * ax
    # +x (value -0.3): diffusion and outflow (u_x > 0 leaves with T_C)
    flux += np.sum(2 * k[:, :, -1] * (-0.3 - T0[:, :, -1])) * ax / h[0] - u[0] * np.sum(T0[:, :, -1]) * ax
    # -y (value 1.5): diffusion and outflow (u_y < 0 leaves through -y with T_C)
    flux += np.sum(2 * k[:, 0, :] * (1.5 - T0[:, 0, :])) * ay / h[1] + u[1] * np.sum(T0[:, 0, :]) * ay
    dE = oracle.total_heat(T1, h) - oracle.total_heat(T0, h)
    assert abs(dE - dt * flux) < 1e-12 * max(1.0, abs(dt * flux))

def test_maximum_principle():
    rng = np.random.default_rng(8)
    shape = (12, 10, 8)
    k = np.exp(0.5 * rng.standard_normal(shape[::-1]))
    bc = _bc([D, D, D, ZF, P, P], [0.2, 0.9, 0.5, 0, 0, 0])
    dt = oracle.dt_max(shape=shape, k=k, bc=bc)   # the limit itself is allowed
    T0 = rng.uniform(0.1, 0.95, shape[::-1])
    T = oracle.run(T0, 80, shape=shape, k=k, bc=bc, dt=dt)
    assert T.min() >= 0.1 - 1e-14 and T.max() <= 0.95 + 1e-14
    # periodic upwind advection-diffusion
    u = (0.3, 0.2, -0.1)
    bc = _bc([P] * 6)
    dt = oracle.dt_max(shape=shape, k=k, u=u, bc=bc)
    T = oracle.run(T0, 80, shape=shape, k=k, u=u, bc=bc, dt=dt)
    assert T.min() >= T0.min() - 1e-14 and T.max() <= T0.max() + 1e-14


def test_layered_steady_state():
    # k varies along x only; Dirichlet TL / TR on x, zero-flux on y and z.
    # The flux through the column is q = (TL - TR) / (hx * sum 1/k_i)
    # (half-cell Dirichlet faces plus harmonic-mean faces add up to series
    # resistance), and that profile is a fixed point of the step.
    rng = np.random.default_rng(9)
    nx, ny, nz = 16, 5, 4
    hx = 0.7
    kx = np.exp(0.5 * rng.standard_normal(nx))
    TL, TR = 1.0, 0.25
    q = (TL - TR) / (hx * np.sum(1.0 / kx))
    prof = np.empty(nx)
    prof[0] = TL - q * hx / (2 * kx[0])
    for i in range(nx - 1):
        Kf = 2 * kx[i] * kx[i + 1] / (kx[i] + kx[i + 1])
        prof[i + 1] = prof[i] - q * hx / Kf
    assert abs(prof[-1] - q * hx / (2 * kx[-1]) - TR) < 1e-13
    k = np.broadcast_to(kx, (nz, ny, nx)).copy()
    T0 = np.broadcast_to(prof, (nz, ny, nx)).copy()
    bc = _bc([D, D, ZF, ZF, ZF, ZF], [TL, TR, 0, 0, 0, 0])
    h = (hx, 1.0, 1.0)
    dt = 0.9 * oracle.dt_max(shape=(nx, ny, nz), h=h, k=k, bc=bc)
    T = oracle.run(T0, 50, shape=(nx, ny, nz), h=h, k=k, bc=bc, dt=dt)
    np.testing.assert_allclose(T, T0, rtol=0, atol=1e-13)
    # uniform k reduces to the linear profile TL - (TL - TR)(i + 1/2)/N
    lin = TL - (TL - TR) * (np.arange(nx) + 0.5) / nx
    T0 = np.broadcast_to(lin, (nz, ny, nx)).copy()
    T = oracle.run(T0, 50, shape=(nx, ny, nz), h=h, k=1.0, bc=bc, dt=dt)
    np.testing.assert_allclose(T, T0, rtol=0, atol=1e-13)


# --------------------------------------------------------------------------
# rounding, threads, argument checks
# --------------------------------------------------------------------------
def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    vals = list(rng.standard_normal(2000) * 10.0 ** rng.integers(-30, 30, 2000))
    # exact ties: low 16 bits 0x8000 with both parities of bit 16
    for hi in (0x3f80, 0x3f81, 0xbf80, 0xbf81, 0x0001, 0x7f7f):
        vals.append(np.array([(hi << 16) | 0x8000], dtype=np.uint32).view(np.float32)[0])
    vals += [0.0, -0.0, 1e-40, -3e-39, np.inf, -np.inf]
    x = np.array(vals, dtype=np.float32).astype(np.float64)
    ours = oracle.round_to(x, "bf16")
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ours, ref)
    assert np.isnan(oracle.round_to(np.nan, "bf16"))
    np.testing.assert_array_equal(oracle.round_to(x, "f32"), x)


def test_thread_count_does_not_change_results():
    rng = np.random.default_rng(13)
    shape = (17, 13, 11)
    k = np.exp(0.5 * rng.standard_normal(shape[::-1]))
    bc = _bc([D, ZF, P, P, DC, D], [1, 0, 0, 0, 0.5, 0])
    T0 = rng.uniform(0, 1, shape[::-1])
    kw = dict(shape=shape, k=k, u=(0.1, -0.2, 0.05), bc=bc, dt=0.05)
    a = oracle.run(T0, 7, threads=1, **kw)
    b = oracle.run(T0, 7, threads=3, **kw)
    np.testing.assert_array_equal(a, b)


def test_rejects_half_periodic_axis():
    with pytest.raises(ValueError):
        oracle.run(np.zeros((2, 2, 2)), 1, shape=(2, 2, 2), bc=_bc([P, D, ZF, ZF, ZF, ZF]), dt=0.1)
