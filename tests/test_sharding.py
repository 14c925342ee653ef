"""Instance sharding of a batch across ranks (host logic, two gloo ranks on the CPU): every instance
is owned by exactly one rank, and the gathered results equal an unsharded run in instance order.
The per-instance "solve" is a fake that depends only on the instance (no GPU)."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp

from paper_2501_05110_gb300 import sharding

COUNT = 11


def _fake_solve(i):
    """Stand-in for one instance's CN steps: a state whose length and values depend on i."""
    g = torch.Generator().manual_seed(100 + i)
    return torch.randn(5 + 3 * (i % 4), generator=g, dtype=torch.float64)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = sharding.shard_instances(COUNT, rank, world)
    out = sharding.gather_instance_states([_fake_solve(i) for i in mine], COUNT, rank, world)
    if rank == 0:
        ref = [_fake_solve(i) for i in range(COUNT)]
        q.put(("ok", all(torch.equal(a, b) for a, b in zip(out, ref)) and len(out) == COUNT))
    else:
        q.put(("none", out is None))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_partition_the_instances():
    for world in (1, 2, 3, 8):
        owned = sorted(i for r in range(world) for i in sharding.shard_instances(COUNT, r, world))
        assert owned == list(range(COUNT))
    with pytest.raises(ValueError):
        sharding.shard_instances(COUNT, 2, 2)


def test_two_ranks_gather_equals_unsharded():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res["ok"] is True and res["none"] is True
