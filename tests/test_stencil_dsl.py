"""The expression front end (paper_2209_13768_gb300.stencil): program
analysis and code generation on the CPU (the generated source is compiled
with nvcc here too), the compiled kernels on the GPU against the FP64 oracle
and against numpy evaluations written in this file."""
import numpy as np
import pytest

import oracle
from paper_2209_13768_gb300 import stencil as S


def _heat():
    T, w = S.Field("T"), S.Param("w")
    return T, w, T + w * (T[-1, 0, 0] + T[1, 0, 0] + T[0, -1, 0] + T[0, 1, 0] + T[0, 0, -1] + T[0, 0, 1] - 6 * T)


def test_program_analysis():
    T, w, e = _heat()
    p = S.Program({T: e})
    assert p.fields == ["T"] and p.written == ["T"] and p.params == ["w"] and p.radius == 1
    K = S.Field("K")
    q = S.Program({T: T + K[0, 0, 2] * (T[0, 0, 1] - T)})
    assert q.fields == ["K", "T"] and q.written == ["T"] and q.params == [] and q.radius == 2
    assert S.Program({T: 2 * T}).radius == 0
    # the own row's z neighbours ride in a register window (its segments,
    # x halo included, shift down a plane); other rows load once a plane
    assert p.windows == {"T": (-1, 1)} and q.windows == {"T": (0, 1)}
    assert p.rows[("T", 0, 0)] == (-1, 1) and p.rows[("T", 1, 0)] == (0, 0)
    assert "s_T_p0_m1_p0 = s_T_p0_p0_p0;" in p.source and "s_T_p0_p0_m1 = s_T_p0_p1_m1;" in p.source
    # other rows: a loop-invariant offset from the per-plane pointer, the
    # 4 cells by one 128-bit load, the x halo masked to the row
    assert "const long long ro_m1_p0 = (-1) * sy + (0) * sz;" in p.source
    assert "__ldg(reinterpret_cast<const float4*>(r_))" in p.source and "q_T += sz;" in p.source
    assert "(unsigned)(x0 + (-1)) < (unsigned)nx ? __ldg(r_ + (-1)) : 0.0f" in p.source
    assert p.key != q.key


def test_program_errors():
    T = S.Field("T")
    with pytest.raises(ValueError):
        S.Field("_x")
    with pytest.raises(ValueError):
        S.Param("1a")
    with pytest.raises(IndexError):
        T[5, 0, 0]
    with pytest.raises(IndexError):
        T[1, 0]
    with pytest.raises(ValueError):
        T + float("inf")
    with pytest.raises(TypeError):
        T + "a"
    with pytest.raises(ValueError):
        S.Program({})
    with pytest.raises(ValueError):
        S.Program({T: T, S.Field("T"): T})   # two fields named T
    with pytest.raises(TypeError):
        S.Program({T: 1.0})


def test_generated_source_compiles_for_sm103a():
    # cross-compiles without a GPU: the generated kernel and launcher build
    T, w, e = _heat()
    K = S.Field("K")
    path = S.build(S.Program({T: e + 0.5 * K[0, 1, 0] / (K + 1.0) - (-T[0, 0, 2])}))
    assert path.endswith(".so")


# ------------------------------------------------------------------ GPU ---
@pytest.mark.gpu
def test_heat_matches_oracle_held_cells():
    torch = pytest.importorskip("torch")
    T, w, e = _heat()
    step = S.compile({T: e})
    rng = np.random.default_rng(5)
    shape = (45, 38, 29)   # ragged against the 32 x 8 x 16 blocking
    gam = [0.3, 0.9, 0.1, 0.6, 0.2, 0.8]
    bc = [("dirichlet_cell", g) for g in gam]
    T0 = oracle.run(rng.uniform(0, 1, shape[::-1]), 0, shape=shape, k=1.0, bc=bc, dt=0.1)   # held layers set
    t = torch.tensor(T0.astype(np.float32), device="cuda")
    step.run({"T": t}, steps=60, w=0.1)
    ref = oracle.run(T0, 60, shape=shape, k=1.0, bc=bc, dt=0.1)
    got = t.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-5
    assert step.launches == 60


def _shift(a, dx, dy, dz, R):
    nz, ny, nx = a.shape
    return a[R + dz:nz - R + dz, R + dy:ny - R + dy, R + dx:nx - R + dx]


@pytest.mark.gpu
def test_variable_coefficient_and_radius_two_against_numpy():
    torch = pytest.importorskip("torch")
    T, K, a = S.Field("T"), S.Field("K"), S.Param("a")
    # a 4th-order x second difference with a cell coefficient and a division
    lap = (-T[-2, 0, 0] + 16 * T[-1, 0, 0] - 30 * T + 16 * T[1, 0, 0] - T[2, 0, 0]) / 12.0
    e = T + a * K * lap / (1.0 + K[0, 1, 0]) + 0.01 * (T[0, 0, -1] - T[0, 0, 1])
    step = S.compile({T: e})
    rng = np.random.default_rng(6)
    shape = (40, 21, 19)
    T0 = rng.uniform(0, 1, shape[::-1])
    K0 = rng.uniform(0.5, 1.5, shape[::-1])
    t = torch.tensor(T0.astype(np.float32), device="cuda")
    k = torch.tensor(K0.astype(np.float32), device="cuda")
    step.run({"T": t, "K": k}, steps=5, a=0.05)
    R = 2
    ref = T0.copy()
    for _ in range(5):
        g = lambda A, dx, dy, dz: _shift(A, dx, dy, dz, R)   # noqa: E731
        lap = (-g(ref, -2, 0, 0) + 16 * g(ref, -1, 0, 0) - 30 * g(ref, 0, 0, 0) + 16 * g(ref, 1, 0, 0)
               - g(ref, 2, 0, 0)) / 12.0
        new = ref.copy()
        new[R:-R, R:-R, R:-R] = (g(ref, 0, 0, 0) + 0.05 * g(K0, 0, 0, 0) * lap / (1.0 + g(K0, 0, 1, 0))
                                 + 0.01 * (g(ref, 0, 0, -1) - g(ref, 0, 0, 1)))
        ref = new
    got = t.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-5
    np.testing.assert_array_equal(k.cpu().numpy(), K0.astype(np.float32))   # read-only field untouched


@pytest.mark.gpu
def test_coupled_updates_read_the_old_values():
    torch = pytest.importorskip("torch")
    A, B, c = S.Field("A"), S.Field("B"), S.Param("c")
    step = S.compile({A: A + c * (B - A), B: B + c * (A - B)})   # both from step n (Jacobi)
    rng = np.random.default_rng(7)
    A0 = rng.uniform(0, 1, (8, 9, 10))
    B0 = rng.uniform(0, 1, (8, 9, 10))
    ta = torch.tensor(A0.astype(np.float32), device="cuda")
    tb = torch.tensor(B0.astype(np.float32), device="cuda")
    step.run({"A": ta, "B": tb}, steps=3, c=0.25)
    a, b = A0.copy(), B0.copy()
    for _ in range(3):
        a, b = a + 0.25 * (b - a), b + 0.25 * (a - b)
    np.testing.assert_allclose(ta.cpu().numpy(), a, rtol=0, atol=1e-6)
    np.testing.assert_allclose(tb.cpu().numpy(), b, rtol=0, atol=1e-6)
    np.testing.assert_allclose((ta + tb).cpu().numpy(), A0 + B0, rtol=0, atol=1e-6)   # conserved


@pytest.mark.gpu
def test_run_argument_errors():
    torch = pytest.importorskip("torch")
    T, w, e = _heat()
    step = S.compile({T: e})
    t = torch.zeros((8, 8, 8), device="cuda")
    with pytest.raises(KeyError):
        step.run({"T": t}, steps=1)               # w missing
    with pytest.raises(KeyError):
        step.run({}, steps=1, w=0.1)
    with pytest.raises(TypeError):
        step.run({"T": t.double()}, steps=1, w=0.1)
    with pytest.raises(ValueError):
        step.run({"T": t}, steps=-1, w=0.1)
    step.run({"T": t}, steps=0, w=0.1)            # no-op


@pytest.mark.parametrize("case", ["pointwise", "coupled", "radius3"])
def test_more_programs_cross_compile(case):
    # code generation for a pointwise update (radius 0), two coupled fields
    # with a read-only third, and a radius-3 stencil with every operator
    A, B, K = S.Field("A"), S.Field("B"), S.Field("K")
    a, b = S.Param("a"), S.Param("b")
    if case == "pointwise":
        prog = S.Program({A: a * A * A - b / (1.0 + A)})
        assert prog.radius == 0 and prog.windows == {}
    elif case == "coupled":
        prog = S.Program({A: A + a * K * (B[1, 0, 0] - A), B: B - a * K[0, -1, 0] * (A[0, 0, 1] - B)})
        assert prog.written == ["A", "B"] and prog.fields == ["A", "B", "K"] and prog.params == ["a"]
    else:
        prog = S.Program({A: A + a * (A[3, 0, 0] - A[-3, 0, 0]) / 6.0 - (-A[0, 0, -3] + A[0, 0, 3]) * b
                          + A[0, 2, 1] * A[0, -2, -1]})
        assert prog.radius == 3 and prog.windows == {"A": (-3, 3)}
        assert "s_A_p0_m3_p0" in prog.source and "s_A_p0_p3_p0" in prog.source and ("A", 0, -2) in prog.rows
    assert S.build(prog).endswith(".so")
