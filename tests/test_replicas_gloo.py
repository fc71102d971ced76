"""The multi-process form of bench.py (one replica per rank, no data-path
collective): the slowest rank's time is taken, and the job's throughput is the
steps of all ranks over that time.  Two gloo ranks on CPU."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 180.0][rank]                 # rank 1 is the slow one
    got = bench.max_over_ranks(ms, world, "cpu")
    value = bench.job_throughput(world, 10, got)
    dist.barrier()
    out.put((rank, got, value))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value in res:
        assert got == 180.0
        assert value == pytest.approx(2 * 10 / 0.18)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(42.5, 1, "cpu") == 42.5
    assert bench.job_throughput(1, 50, 100.0) == pytest.approx(500.0)
