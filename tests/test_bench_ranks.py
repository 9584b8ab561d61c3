"""The bench's multi-rank logic on CPU: two gloo ranks (world size 2).

On N GPUs every rank runs its own replica of the workload; the job's step
time is the slowest rank's (a MAX all-reduce after a barrier) and the value
counts the units of all ranks.  The reference arm runs on rank 0 only.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

from tests.conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 1.5 + rank            # rank 1 is the slower one
        dist.barrier()
        got = bench.max_over_ranks(ms, dist, "cpu")
        q.put((rank, got, bench.job_value(world, 3.0e9, got)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_time_and_all_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive and all(p.exitcode == 0 for p in procs)
    out = sorted(q.get(timeout=5) for _ in range(2))
    for rank, got, value in out:
        assert got == 2.5
        assert value == pytest.approx(2 * 3.0e9 / 2.5e-3 / 1e9)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.0, None, "cpu") == 4.0
    assert bench.job_value(1, 4194305 * 1024, 0.5) == pytest.approx(4194305 * 1024 / 0.5e-3 / 1e9)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    bench.run_reference(None, 1, 2)      # rank 1 of 2: no work, no output
    assert capsys.readouterr().out == ""
