"""The seeded input recipes (CPU): shapes, distributions and determinism of
the synthetic workloads the benchmark and the tests use."""
import numpy as np

from paper_2209_13768_gb300 import workloads as W


def test_seeded_fields_are_deterministic_and_distributed():
    a = W.uniform01((33, 17, 9), 3)
    assert a.dtype == np.float32 and a.shape == (9, 17, 33)
    np.testing.assert_array_equal(a, W.uniform01((33, 17, 9), 3))
    assert 0.0 <= a.min() and a.max() < 1.0 and abs(a.mean() - 0.5) < 0.02
    k = W.lognormal_k((64, 64, 32), 2)
    z = np.log(k.astype(np.float64))
    assert k.min() > 0 and abs(z.mean()) < 0.01 and abs(z.std() - 0.5) < 0.01


def test_paper_workload_settings():
    p = W.heat_64()
    assert p.shape == (64, 64, 64) and p.k == 1.0 and p.steps == 100
    q = W.implicit_problem((16, 16, 16))
    assert q.dt == 0.1 and q.k == 1.0 and q.bc[0] == ("dirichlet_cell", 1.0)
    assert all(b == ("dirichlet_cell", 0.0) for b in q.bc[1:])   # omega = k dt / h^2 = 1/10, held layers
    r = W.heat_lognormal((32, 32, 32), steps=7)
    assert r.bc[0] == ("dirichlet", 1.0) and r.bc[1] == ("dirichlet", 0.0) and r.steps == 7
    a = W.advection_diffusion((64, 64, 32), steps=3)
    assert a.u == (0.3, 0.1, 0.05) and a.dt == 1.0 and a.bc[0][0] == "periodic"
    assert np.unravel_index(np.argmax(a.T0), a.T0.shape) == (16, 32, 32)   # blob at the centre (z, y, x)


def test_batch_grids_recipe():
    gs = W.batch_grids(count=256)
    edges = np.array([g.shape for g in gs])
    steps = np.array([g.steps for g in gs])
    assert edges.min() >= 16 and edges.max() <= 128
    # log-uniform edges: log(edge) spread evenly over [log 16, log 128]
    le = np.log(edges.ravel())
    assert abs(le.mean() - 0.5 * (np.log(16) + np.log(128))) < 0.08
    assert steps.min() >= 50 and steps.max() <= 500 and abs(steps.mean() - 275) < 25
    assert all(g.bc == [("dirichlet", 0.0)] * 6 for g in gs)
    assert [g.shape for g in W.batch_grids(count=256)] == [g.shape for g in gs]   # seeded


def test_request_stream_recipe():
    arr = W.request_stream(rate=200.0, count=2000, pool=8)
    t = np.array([a.t for a in arr])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0            # Poisson: exponential gaps, mean 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    edges = np.array([a.problem.shape for a in arr[:8]])
    assert edges.min() >= 32 and edges.max() <= 256
    steps = np.array([a.problem.steps for a in arr])
    assert steps.min() >= 50 and steps.max() <= 2000
    st = np.array([a.storage for a in arr])
    assert abs(st.mean() - 0.5) < 0.05
    assert arr[8].problem.shape == arr[0].problem.shape            # the pool of 8 shapes is reused
