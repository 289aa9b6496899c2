"""Batched persistent launch and the continuous-batching server (GPU).

Both run the same per-cell arithmetic as wfa_step, so every result must be
bit-identical to the grid advanced alone."""
import os
import time

import numpy as np
import pytest

import paper_2209_13768_gb300 as wfa
from paper_2209_13768_gb300 import workloads as W
from helpers import make_grid, rel_linf, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

D, ZF, P, DC = W.D, W.ZF, W.P, W.DC


def _problem(i, rng):
    shape = tuple(int(v) for v in rng.integers(5, 70, 3))
    nx, ny, nz = shape
    mixes = [[(D, 0.5)] * 6, [(P, 0)] * 2 + [(ZF, 0)] * 4, [(DC, 1.0), (D, 0.0), (P, 0), (P, 0), (ZF, 0), (D, 0.3)]]
    kvar = i % 2 == 0
    k = np.exp(0.5 * rng.standard_normal((nz, ny, nx))).astype(np.float32) if kvar else 0.7
    u = tuple(rng.uniform(-0.3, 0.3, 3)) if i % 3 == 0 else (0.0, 0.0, 0.0)
    T0 = rng.uniform(0, 1, (nz, ny, nx)).astype(np.float32)
    return W.Problem(shape=shape, T0=T0, k=k, u=u, bc=mixes[i % 3], steps=int(rng.integers(0, 40)))


def test_batch_bitwise_equals_solo():
    rng = np.random.default_rng(42)
    probs = [_problem(i, rng) for i in range(14)]
    storages = [wfa.BF16 if i % 4 == 1 else wfa.F32 for i in range(len(probs))]
    grids = [make_grid(p, storage=s) for p, s in zip(probs, storages)]
    try:
        wfa.batch_run(grids, [p.steps for p in probs])
        for p, s, g in zip(probs, storages, grids):
            assert g.steps_done() == p.steps
            solo = run_gpu(p, storage=s, variant=-1)
            np.testing.assert_array_equal(g.read_field(), solo, err_msg=f"{p.shape} steps {p.steps}")
        # a second batch continues from where the first stopped
        wfa.batch_run(grids, [3] * len(grids))
        for p, s, g in zip(probs, storages, grids):
            np.testing.assert_array_equal(g.read_field(), run_gpu(p, steps=p.steps + 3, storage=s, variant=-1))
    finally:
        for g in grids:
            g.close()


def test_batch_matches_oracle():
    rng = np.random.default_rng(7)
    probs = W.batch_grids(count=12, lo=16, hi=48, seed=9, steps=(5, 30))
    grids = [make_grid(p) for p in probs]
    try:
        wfa.batch_run(grids, [p.steps for p in probs])
        for p, g in zip(probs, grids):
            assert rel_linf(g.read_field(), run_oracle(p)) <= 1e-5
    finally:
        for g in grids:
            g.close()


def test_batch_sizes_steps_and_classes():
    # tiny and large grids, zero and single steps, every class of the batched
    # sweep (f32 / bf16, uniform / per-cell k, advection, ghost-layer faces)
    rng = np.random.default_rng(17)
    shapes = [(2, 2, 2), (3, 5, 2), (130, 67, 40), (16, 16, 16), (9, 70, 5), (64, 8, 33)]
    mixes = [[(D, 0.5)] * 6, [(D, 0.25), (ZF, 0), (ZF, 0), (D, -0.5), (ZF, 0), (D, 1.0)],
             [(P, 0)] * 2 + [(ZF, 0)] * 4, [(DC, 1.0)] + [(D, 0.0)] * 5]
    probs, storages = [], []
    for i in range(24):
        shape = shapes[i % len(shapes)]
        nx, ny, nz = shape
        mix = mixes[(i // 2) % len(mixes)]
        if any(k == DC for k, _ in mix) and min(shape) < 3:
            mix = mixes[0]
        kvar = i % 3 != 0
        k = np.exp(0.5 * rng.standard_normal((nz, ny, nx))).astype(np.float32) if kvar else 0.6
        u = tuple(rng.uniform(-0.3, 0.3, 3)) if i % 4 == 1 else (0.0, 0.0, 0.0)
        T0 = rng.uniform(0, 1, (nz, ny, nx)).astype(np.float32)
        probs.append(W.Problem(shape=shape, T0=T0, k=k, u=u, bc=mix, steps=[0, 1, 2, 7, 23, 40][i % 6]))
        storages.append(wfa.BF16 if i % 5 == 2 else wfa.F32)
    grids = [make_grid(p, storage=s) for p, s in zip(probs, storages)]
    try:
        wfa.batch_run(grids, [p.steps for p in probs])
        for p, s, g in zip(probs, storages, grids):
            assert g.steps_done() == p.steps
            np.testing.assert_array_equal(g.read_field(), run_gpu(p, storage=s, variant=-1),
                                          err_msg=f"{p.shape} steps {p.steps} storage {s}")
    finally:
        for g in grids:
            g.close()


def test_batch_modes_agree_bitwise():
    # the persistent kernel, per-round launches in a graph, and on the stream: the same fields
    rng = np.random.default_rng(23)
    probs = [_problem(i, rng) for i in range(12)]
    outs = []
    for mode in ("persistent", "rounds", "stream"):
        os.environ["WFA_BATCH_MODE"] = mode
        try:
            grids = [make_grid(p) for p in probs]
            wfa.batch_run(grids, [p.steps for p in probs])
            outs.append([g.read_field() for g in grids])
            for g in grids:
                g.close()
        finally:
            os.environ.pop("WFA_BATCH_MODE", None)
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            np.testing.assert_array_equal(a, b)


def test_batch_wait_times_out_cleanly():
    # a barrier target that no arrival satisfies (host-side test hook): the
    # bounded device wait gives up, the call reports it, the context lives on
    p = _problem(0, np.random.default_rng(3))
    p.steps = 4
    g = make_grid(p)
    try:
        os.environ["WFA_TEST_BATCH_STALL"] = "1"
        os.environ["WFA_BATCH_MODE"] = "persistent"   # the mode with a device-side wait
        t0 = time.time()
        with pytest.raises(wfa.WfaError) as e:
            wfa.batch_run([g], [4])
        assert e.value.code == -6
        assert time.time() - t0 < 30
    finally:
        os.environ.pop("WFA_TEST_BATCH_STALL", None)
        os.environ.pop("WFA_BATCH_MODE", None)
        g.close()
    q = _problem(1, np.random.default_rng(4))
    q.steps = 5
    with make_grid(q) as g2:
        wfa.batch_run([g2], [5])
        np.testing.assert_array_equal(g2.read_field(), run_gpu(q, variant=-1))


def test_server_results_equal_alone_and_in_a_mix():
    rng = np.random.default_rng(11)
    probs = [_problem(i, rng) for i in range(10)]
    for p in probs:
        p.steps = max(p.steps, 1)
    storages = [wfa.BF16 if i % 3 == 2 else wfa.F32 for i in range(len(probs))]
    with wfa.Server(budget_bytes=4 << 30, quantum=7) as srv:
        tickets = []
        for i, (p, s) in enumerate(zip(probs, storages)):
            tickets.append(srv.submit(p.shape, p.T0, p.steps, h=p.h, storage=s, k=p.k, u=p.u, bc=p.bc))
            if i % 3 == 0:
                time.sleep(0.01)   # arrivals while others are running
        outs = [srv.wait(t, timeout=60) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(probs) and st["rejected"] == 0
    assert st["p99_latency_s"] >= st["p50_latency_s"] > 0
    for p, s, out in zip(probs, storages, outs):
        np.testing.assert_array_equal(out, run_gpu(p, storage=s, variant=-1))


def test_server_budget_admission():
    # a request larger than the budget is refused at submission; requests that
    # fit only one at a time still all complete (admitted as memory frees up)
    rng = np.random.default_rng(5)
    p = _problem(2, rng)
    p.shape = (40, 40, 40)
    p.T0 = rng.uniform(0, 1, (40, 40, 40)).astype(np.float32)
    p.k = 1.0
    p.steps = 6
    with wfa.Server(budget_bytes=1 << 20) as srv:
        with pytest.raises(wfa.WfaError) as e:
            srv.submit(p.shape, p.T0, p.steps, bc=p.bc)
        assert e.value.code == -8
    one = 2 * (64 * 56 * 56 * 4) + 40 ** 3 * 4 + 65536
    with wfa.Server(budget_bytes=int(one * 1.5), quantum=2) as srv:
        tickets = [srv.submit(p.shape, p.T0, p.steps, bc=p.bc) for _ in range(4)]
        outs = [srv.wait(t, timeout=60) for t in tickets]
        st = srv.stats()
    assert st["peak_resident_bytes"] <= int(one * 1.5)
    ref = run_gpu(p, variant=-1)
    for out in outs:
        np.testing.assert_array_equal(out, ref)


def test_server_request_fails_cleanly_on_injected_oom():
    # the first device allocation of some request fails (host-side
    # injection): that request alone reports the error, the others complete
    # bitwise, and the server's memory accounting returns to zero
    rng = np.random.default_rng(17)
    probs = [_problem(i, rng) for i in range(6)]
    for p in probs:
        p.steps = max(p.steps, 2)
    try:
        with wfa.Server(budget_bytes=4 << 30, quantum=5) as srv:
            wfa.inject_alloc_failure(0)
            tickets = [srv.submit(p.shape, p.T0, p.steps, h=p.h, k=p.k, u=p.u, bc=p.bc) for p in probs]
            outs, failed = [], 0
            for t in tickets:
                try:
                    outs.append(srv.wait(t, timeout=60))
                except wfa.WfaError as e:
                    assert "out of memory" in str(e)
                    outs.append(None)
                    failed += 1
            st = srv.stats()
    finally:
        wfa.inject_alloc_failure(-1)
    assert failed == 1 and st["completed"] == len(probs) - 1
    assert st["resident_bytes"] == 0
    for p, out in zip(probs, outs):
        if out is not None:
            np.testing.assert_array_equal(out, run_gpu(p, variant=-1))
