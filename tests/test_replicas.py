"""Replicas on several GPUs: host logic of the timed region on CPU ranks.

The compact step does not shard (every replica runs the whole workload on
its own GPU), so a multi-GPU run is N independent replicas; the only
collectives are the barrier around the timed region and the max over ranks
of its duration.  Here two gloo ranks on the CPU stand in for two GPUs.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.replica_max(100.0 + 50.0 * rank, world, torch.device("cpu"))
        value = bench.job_value(59049, 100, 5, ms, world)
        q.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want_ms = 150.0
    for rank, ms, value in out:
        assert ms == want_ms
        assert value == pytest.approx(world * 59049 * 100 * 5 / (want_ms / 1e3))


def test_single_rank_needs_no_collective():
    assert bench.replica_max(12.5, 1, None) == 12.5
    assert bench.job_value(10, 100, 2, 1000.0, 1) == pytest.approx(2000.0)
