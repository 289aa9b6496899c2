"""The oracle's pins are sharp: each plausible mistake planted in a copy of the
oracle source (on the CPU, in a temporary build) fails at least one of them."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from test_oracle_implicit import dense_implicit
from test_oracle_pins import BC_MIXES, _apply_held, _bc, brute_matrix, _spectral_solution

SRC = os.path.join(os.path.dirname(oracle.__file__), "wfa_oracle.c")

MUTANTS = {
    "flux sign at the upper cell": ("acc[D] += -diff + F;", "acc[D] += diff + F;"),
    "upwind operands swapped": ("const double F = (up * T[C] + um * T[D]) * inv_h;",
                                "const double F = (up * T[D] + um * T[C]) * inv_h;"),
    "half-cell Dirichlet factor dropped": ("2.0 * kc(p, C0) * (vlo - T[C0])",
                                           "1.0 * kc(p, C0) * (vlo - T[C0])"),
    "arithmetic instead of harmonic mean": ("return s > 0.0 ? 2.0 * a * b / s : 0.0;",
                                            "return 0.5 * s;"),
    "periodic wrap face dropped": ("periodic ? (na > 1 ? na : 0) : na - 1;", "na - 1;"),
    "upper outflow sign": ("acc[C1] += diff - F;", "acc[C1] += diff + F;"),
    "spacing of the wrong axis": ("const double inv_h2 = 1.0 / (p->h[a] * p->h[a]);",
                                  "const double inv_h2 = 1.0 / (p->h[b] * p->h[b]);"),
    "held cells updated": ("if (held[c]) continue;", "(void)0;"),
    "dt limit without the Dirichlet factor": ("D += 2.0 * kc(&p, C) * inv_h2;",
                                              "D += kc(&p, C) * inv_h2;"),
    "dt limit without advection": ("if (side == 1 && u[a] > 0.0) D += u[a] / h[a];", ""),
    "CG without beta (steepest descent)": ("const double beta = rr_new / rr;", "const double beta = 0.0;"),
    "implicit right-hand side without boundary terms": ("r[c] = held[c] ? 0.0 : T[c] + dt * acc[c];\n            x[c]",
                                                        "r[c] = held[c] ? 0.0 : T[c];\n            x[c]"),
    "implicit operator sign": ("out[c] = held[c] ? 0.0 : y[c] - p0->dt * acc[c];",
                               "out[c] = held[c] ? 0.0 : y[c] + p0->dt * acc[c];"),
    "CG residual update sign": ("r[c] -= alpha * q[c];", "r[c] += alpha * q[c];"),
    "Dirichlet values left in the linear part": ("for (int f = 0; f < 6; ++f) p0.value[f] = 0.0;\n#ifdef _OPENMP\n    if (nthreads > 0) omp_set_num_threads(nthreads);\n#else\n    (void)nthreads;\n#endif\n    const int64_t N = n[0] * n[1] * n[2];\n    unsigned char* held = held_mask(&p);\n    double* buf = (double*)malloc((size_t)N * 6",
                                                 "(void)0;\n#ifdef _OPENMP\n    if (nthreads > 0) omp_set_num_threads(nthreads);\n#else\n    (void)nthreads;\n#endif\n    const int64_t N = n[0] * n[1] * n[2];\n    unsigned char* held = held_mask(&p);\n    double* buf = (double*)malloc((size_t)N * 6"),
    "implicit held cells overwritten": ("if (!held[c]) T[c] = x[c];\n        total += it;\n        last = bb > 0.0 ? sqrt(rr / bb)",
                                        "T[c] = x[c];\n        total += it;\n        last = bb > 0.0 ? sqrt(rr / bb)"),
    "CG-CG step length without its beta correction": ("const double den = delta - beta * g1 / alpha;",
                                                      "const double den = delta;"),
    "CG-CG A p recurrence without beta": ("sv[c] = w[c] + beta * sv[c];", "sv[c] = w[c];"),
}


def battery(lib):
    """Run a compact set of pins against one oracle build; return the failures."""
    failed = []
    # brute-force matrix, every feature at once
    rng = np.random.default_rng(101)
    shape = (4, 3, 5)
    nx, ny, nz = shape
    for mix in (BC_MIXES[4], BC_MIXES[6], BC_MIXES[2]):
        k = np.exp(0.5 * rng.standard_normal((nz, ny, nx)))
        u = (0.3, -0.2, 0.25)
        h = (1.1, 0.8, 1.3)
        bc = _bc(mix, list(rng.uniform(-1, 2, 6)))
        try:
            dtm = oracle.dt_max(shape=shape, h=h, k=k, u=u, bc=bc, lib=lib)
            M, b, held = brute_matrix(shape, h, k, u, bc, 0.9 * dtm)
            T0 = _apply_held(rng.uniform(0, 1, (nz, ny, nx)), shape, held)
            T = oracle.run(T0, 3, shape=shape, h=h, k=k, u=u, bc=bc, dt=0.9 * dtm, lib=lib)
            ref = T0.ravel()
            for _ in range(3):
                ref = M @ ref + b
            if not np.allclose(T.ravel(), ref, rtol=0, atol=1e-12):
                failed.append("brute")
            M1, _, _ = brute_matrix(shape, h, k, u, bc, dtm)
            M2, _, _ = brute_matrix(shape, h, k, u, bc, 1.02 * dtm)
            if M1.min() < -1e-13 or M2.min() > -1e-6:
                failed.append("dt limit")
        except ValueError:
            failed.append("rejected")
    # paper omega
    if abs(oracle.dt_max(shape=(8, 8, 8), k=1.0, bc=_bc(["dirichlet"] * 6), lib=lib) - 1 / 9) > 1e-15:
        failed.append("omega")
    # spectral whole field
    shape = (10, 9, 7)
    kinds = ("periodic", "zeroflux", "dirichlet")
    bc = _bc([kinds[0]] * 2 + [kinds[1]] * 2 + [kinds[2]] * 2)
    u = (0.4, 0, 0)
    T0 = np.random.default_rng(11).uniform(0, 1, shape[::-1])
    T = oracle.run(T0, 10, shape=shape, h=(1.0, 0.9, 1.2), k=0.6, u=u, bc=bc, dt=0.2, lib=lib)
    ref = _spectral_solution(T0, 10, shape, (1.0, 0.9, 1.2), 0.6, u, kinds, 0.2)
    if not np.allclose(T, ref, rtol=0, atol=1e-12):
        failed.append("spectral")
    # implicit step: dense solve, and the CG iteration bound
    rng = np.random.default_rng(102)
    shape = (5, 4, 6)
    k = np.exp(0.5 * rng.standard_normal(shape[::-1]))
    for mix in (BC_MIXES[4], BC_MIXES[5]):
        bc = _bc(mix, list(rng.uniform(-1, 2, 6)))
        T0 = rng.uniform(0, 1, shape[::-1])
        try:
            T, _, _ = oracle.implicit(T0, 2, shape=shape, h=(1.1, 0.8, 1.3), k=k, bc=bc, dt=0.7, rtol=1e-14,
                                      max_iter=2000, lib=lib)
            ref, _, _ = dense_implicit(T0, 2, shape, (1.1, 0.8, 1.3), k, bc, 0.7)
            if not np.allclose(T, ref, rtol=0, atol=1e-10):
                failed.append("implicit dense")
        except ValueError:
            failed.append("implicit rejected")
    shape = (5, 4, 4)
    bc = _bc(["dirichlet_cell"] * 2 + ["periodic"] * 4)
    T0 = np.random.default_rng(4).uniform(0, 1, shape[::-1])
    _, iters, res = oracle.implicit(T0, 1, shape=shape, k=1.0, bc=bc, dt=0.9, rtol=1e-12, max_iter=2000, lib=lib)
    if iters > 15 or res > 1e-12:   # 15 distinct eigenvalues
        failed.append("implicit iterations")
    # Chronopoulos-Gear CG: the iterates of classic CG
    rng = np.random.default_rng(103)
    shape = (7, 5, 6)
    k = np.exp(0.5 * rng.standard_normal(shape[::-1]))
    bc = _bc(BC_MIXES[4], list(rng.uniform(-1, 2, 6)))
    T0 = rng.uniform(0, 1, shape[::-1])
    try:
        for m in (2, 5, 9):
            a, _, _ = oracle.implicit(T0, 1, shape=shape, k=k, bc=bc, dt=2.0, rtol=0.0, max_iter=m, lib=lib)
            b, _, _ = oracle.implicit(T0, 1, shape=shape, k=k, bc=bc, dt=2.0, rtol=0.0, max_iter=m, lib=lib,
                                      method="cgcg")
            if not np.allclose(a, b, rtol=0, atol=1e-12):
                failed.append("cgcg iterates")
                break
    except ValueError:
        failed.append("cgcg rejected")
    return failed


def _build_variant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not found exactly once"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "mut.so"
    subprocess.run(["gcc", "-O1", "-shared", "-fPIC", "-std=c11", str(path), "-o", str(so), "-lm"],
                   check=True, capture_output=True)
    return oracle._bind(str(so))


def test_unmutated_passes_battery():
    assert battery(oracle._load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    lib = _build_variant(tmp_path, name, *MUTANTS[name])
    failures = battery(lib)
    if name == "held cells updated":
        T = oracle.run(np.zeros((4, 4, 4)), 1, shape=(4, 4, 4), k=1.0,
                       bc=_bc(["dirichlet_cell"] * 6, [1.0] * 6), dt=0.1, lib=lib)
        if T[0, 0, 0] != 1.0:
            failures.append("held")
    assert failures, f"mutant {name!r} passed every pin"
