"""Multi-rank bench logic on CPU ranks (gloo, world size 2): replicas time
themselves, the job time is the slowest rank's, the rate counts every rank's
updates, and only rank 0 runs the oracle's reference arm."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times = [0.5, 2.0]                    # rank 1 is the slow replica
        t = bench.max_over_ranks(times[rank], dist, "cpu")
        rate = bench.job_rate(world, 1e9, t)  # 1e9 updates per rank
        out.put((rank, t, rate))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_rate_counts_all_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == 2.0
        assert rate == pytest.approx(world * 1e9 / 2.0 / 1e9)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_rate(1, 2e9, 2.0) == pytest.approx(1.0)


def test_reference_arm_runs_on_rank_zero_only():
    class Args:
        workload, solve_steps, shape, steps, warmup, gpus = "lognormal", 0, "", 1, 0, 2
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(Args, rank=1)
    assert buf.getvalue() == ""
