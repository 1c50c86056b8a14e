"""bench.py's multi-GPU contract on the host, with two gloo ranks on CPU:
every rank runs the same replica workload, the timed region is the maximum
over the ranks, the value counts every rank's units, and only rank 0 runs
the reference arm (the others return without work)."""

from __future__ import annotations

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r reports (r + 1, 10 - r) ms: the maxima are (world, 10)
        got = bench.max_over_ranks([rank + 1.0, 10.0 - rank], "cpu")
        dist.barrier()
        ref = bench.run_reference(type("A", (), {"workload": "conv1", "warmup": 0, "steps": 1})(), rank, world)
        q.put((rank, got, ref is None))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_only_rank0_runs_the_reference():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, got, no_ref in res:
        assert got == [2.0, 10.0]
        assert no_ref == (rank != 0)


def test_whole_job_rate_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench
    # 20 layers per step, 100 steps, 4 replicas, 10 ms for the slowest rank
    assert bench.whole_job_rate(20, 100, 4, 10.0) == pytest.approx(20 * 100 * 4 / 0.010)
