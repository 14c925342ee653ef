"""Host logic of bench.py's multi-process path (one process per GPU, replicas of the workload): the
job time is the slowest rank's, the value counts every rank's work.  Run as two gloo ranks on the
CPU; no GPU is used."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank, world, device="cpu")  # rank 1 is the slow one
    q.put((rank, t, bench.job_value(1000, 4, world, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 2.0, (rank, t)
        assert v == pytest.approx(1000 * 4 * 2 / 2.0)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_value(10, 2, 1, 4.0) == 5.0
