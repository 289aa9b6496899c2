"""Seeded synthetic inputs with the shapes and distributions of the paper's
workloads (uniform Cartesian grids, omega = 1/10, Sec. 1.1.1 and Sec. 3.1) and
of the benchmark configurations built on them. The paper uses no dataset; these
stand in for its heat-equation test problems.

Only input generation lives here (random fields, conductivities, boundary
choices, request streams). Nothing in this module evaluates the method: both
the oracle and the CUDA library consume these inputs independently.
Arrays are float32, indexed [z, y, x].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

D, ZF, P, DC = "dirichlet", "zeroflux", "periodic", "dirichlet_cell"


@dataclass
class Problem:
    shape: tuple                      # (nx, ny, nz)
    T0: np.ndarray                    # (nz, ny, nx) float32
    k: object = 1.0                   # scalar or (nz, ny, nx) float32
    u: tuple = (0.0, 0.0, 0.0)
    bc: list = field(default_factory=lambda: [(ZF, 0.0)] * 6)
    h: tuple = (1.0, 1.0, 1.0)
    dt: float = 0.0                   # 0: 0.9 x the stability limit
    dt_factor: float = 0.9
    steps: int = 1
    name: str = ""


def uniform01(shape, seed):
    nx, ny, nz = shape
    return np.random.default_rng(seed).random((nz, ny, nx), dtype=np.float32)


def lognormal_k(shape, seed, sigma=0.5):
    nx, ny, nz = shape
    z = np.random.default_rng(seed).standard_normal((nz, ny, nx), dtype=np.float32)
    return np.exp(np.float32(sigma) * z).astype(np.float32)


def gaussian_blob(shape, centre, sigma):
    """exp(-|x - c|^2 / (2 sigma^2)) at cell centres, c in cell-index units."""
    nx, ny, nz = shape
    x = (np.arange(nx, dtype=np.float32) - np.float32(centre[0])) ** 2
    y = (np.arange(ny, dtype=np.float32) - np.float32(centre[1])) ** 2
    z = (np.arange(nz, dtype=np.float32) - np.float32(centre[2])) ** 2
    s = np.float32(2.0 * sigma * sigma)
    return (np.exp(-z / s)[:, None, None] * np.exp(-y / s)[None, :, None]
            * np.exp(-x / s)[None, None, :]).astype(np.float32)


def heat_64(held_cells=False):
    """64^3, k = 1, T = 0 on every face, T0 ~ U[0,1) (seed 1), 100 steps.
    held_cells: the paper's own boundary (outer cell layer held at 0)."""
    shape = (64, 64, 64)
    return Problem(shape=shape, T0=uniform01(shape, 1), k=1.0,
                   bc=[(DC if held_cells else D, 0.0)] * 6, steps=100,
                   name="heat 64^3 " + ("held cells" if held_cells else "face Dirichlet"))


def heat_lognormal(shape=(512, 512, 512), steps=1000):
    """Per-cell k ~ lognormal(0, 0.5) (seed 2), x faces Dirichlet 1 / 0, y and z
    zero-flux, T0 ~ U[0,1) (seed 3). Default: 512^3, 1000 steps."""
    return Problem(shape=shape, T0=uniform01(shape, 3), k=lognormal_k(shape, 2),
                   bc=[(D, 1.0), (D, 0.0), (ZF, 0.0), (ZF, 0.0), (ZF, 0.0), (ZF, 0.0)],
                   steps=steps, name="heat lognormal k %dx%dx%d" % shape)


def advection_diffusion(shape=(1024, 1024, 512), steps=500):
    """k = 0.05, u = (0.3, 0.1, 0.05) cells per step, dt = 1, periodic x,
    zero-flux y and z, Gaussian blob (sigma = 32 cells) at the grid centre."""
    nx, ny, nz = shape
    sigma = 32.0 * min(nx, ny, nz) / 512.0 if min(nx, ny, nz) < 512 else 32.0
    return Problem(shape=shape, T0=gaussian_blob(shape, (nx / 2, ny / 2, nz / 2), sigma), k=0.05,
                   u=(0.3, 0.1, 0.05), bc=[(P, 0.0)] * 2 + [(ZF, 0.0)] * 4, dt=1.0, steps=steps,
                   name="advection-diffusion %dx%dx%d" % shape)


IMPLICIT_SHAPE = (512, 512, 512)


def implicit_problem(shape=IMPLICIT_SHAPE, steps=10, lognormal=False):
    """The implicit workload (Sec. 1.1.2, Eq. impl_form): k = 1, h = 1,
    omega = k dt / h^2 = 1/10 (dt = 0.1, the paper's testing value), outer cell
    layers held (-x at 1, the other faces at 0), T0 ~ U[0,1) (seed 3).
    lognormal: per-cell k ~ lognormal(0, 0.5) (seed 2) instead, same dt."""
    k = lognormal_k(shape, 2) if lognormal else 1.0
    return Problem(shape=shape, T0=uniform01(shape, 3), k=k, bc=[(DC, 1.0)] + [(DC, 0.0)] * 5, dt=0.1,
                   steps=steps, name="implicit CG %s%dx%dx%d" % (("lognormal k " if lognormal else ""), *shape))


def batch_grids(count=256, lo=16, hi=128, seed=4, steps=(50, 500)):
    """count grids, every edge log-uniform in [lo, hi], k ~ lognormal(0, 0.5),
    T = 0 on every face, T0 ~ U[0,1), steps uniform in [steps[0], steps[1]]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        edges = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), 3))).astype(int)
        shape = tuple(int(e) for e in edges)
        n = int(rng.integers(steps[0], steps[1] + 1))
        s = int(rng.integers(0, 2**31))
        out.append(Problem(shape=shape, T0=uniform01(shape, s), k=lognormal_k(shape, s + 1),
                           bc=[(D, 0.0)] * 6, steps=n, name=f"batch grid {i}"))
    return out


@dataclass
class Arrival:
    t: float           # seconds after the start
    problem: Problem
    storage: int       # 0 fp32, 1 bf16


@dataclass
class RequestSpec:
    """One arrival of the request stream before its fields exist (they are
    drawn from their own seed when the request is made)."""
    t: float
    shape: tuple
    steps: int
    seed: int
    heat: bool
    storage: int


def request_specs(rate=200.0, count=10000, lo=32, hi=256, steps=(50, 2000), seed=5, duration=None):
    """The arrivals of request_stream without their fields: Poisson arrival
    times (mean `rate` per second), edges log-uniform in [lo, hi], steps
    uniform in [steps[0], steps[1]], heat or advection-diffusion and fp32 or
    bf16 with probability 1/2 each. Cheap for long streams (10^4 requests)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while len(out) < count:
        t += rng.exponential(1.0 / rate)
        if duration is not None and t > duration:
            break
        edges = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), 3))).astype(int)
        shape = tuple(int(e) for e in edges)
        n = int(rng.integers(steps[0], steps[1] + 1))
        s = int(rng.integers(0, 2**31))
        heat = bool(rng.random() < 0.5)
        storage = int(rng.random() < 0.5)
        out.append(RequestSpec(t=t, shape=shape, steps=n, seed=s, heat=heat, storage=storage))
    return out


def make_request(spec):
    """The Problem of one request: heat (lognormal k, T = 0 on every face,
    T0 ~ U[0,1)) or advection-diffusion (k = 0.05, u = (0.3, 0.1, 0.05),
    periodic x, zero-flux y / z, a Gaussian blob), fields from its seed."""
    shape, s = spec.shape, spec.seed
    if spec.heat:
        return Problem(shape=shape, T0=uniform01(shape, s), k=lognormal_k(shape, s + 1), bc=[(D, 0.0)] * 6,
                       steps=spec.steps, name="heat")
    nx, ny, nz = shape
    return Problem(shape=shape, T0=gaussian_blob(shape, (nx / 2, ny / 2, nz / 2), max(2.0, min(shape) / 16)),
                   k=0.05, u=(0.3, 0.1, 0.05), bc=[(P, 0.0)] * 2 + [(ZF, 0.0)] * 4, dt=1.0, steps=spec.steps,
                   name="advection-diffusion")


def request_stream(rate=200.0, count=10000, lo=32, hi=256, steps=(50, 2000), seed=5, duration=None, pool=None):
    """Poisson arrivals (mean `rate` per second) of heat or advection-diffusion
    solves (probability 1/2 each), edges log-uniform in [lo, hi], steps uniform
    in [steps[0], steps[1]], fp32 or bf16 storage (probability 1/2 each).
    pool: only the first `pool` arrivals get their own fields; arrival i
    reuses the shape and fields of arrival i % pool (its time, step count and
    storage stay its own), so long streams need little host memory."""
    from dataclasses import replace

    out = []
    for spec in request_specs(rate, count, lo, hi, steps, seed, duration):
        if pool is not None and len(out) >= pool:
            prob = replace(out[len(out) % pool].problem, steps=spec.steps)
        else:
            prob = make_request(spec)
        out.append(Arrival(t=spec.t, problem=prob, storage=spec.storage))
    return out
