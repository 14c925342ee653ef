"""Sharding of independent problem instances across ranks (one process per GPU).

A batch of independent shock instances has no exchange between instances: rank r solves the
instances i with i mod world == r as its own batch, and only the results are gathered.  The
instance order of the gathered state is the order of the unsharded batch.
"""
from __future__ import annotations


def shard_instances(count: int, rank: int, world: int) -> list:
    """Instance indices owned by `rank` (round robin, so every rank gets a similar l_max mix)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return list(range(rank, count, world))


def gather_instance_states(local_states, count: int, rank: int, world: int, dst: int = 0):
    """Gather per-instance state tensors (CPU or device) from every rank to rank `dst`.

    ``local_states`` are the states of this rank's instances, in shard order.  Returns, on `dst`, the
    list of all `count` instance states in global instance order (CPU tensors); None elsewhere.  Uses
    one object gather (the results only: no collective on the solve path)."""
    import torch.distributed as dist
    mine = shard_instances(count, rank, world)
    if len(local_states) != len(mine):
        raise ValueError("one state per owned instance expected")
    payload = [(i, s.detach().cpu()) for i, s in zip(mine, local_states)]
    if world == 1:
        return [s for _, s in sorted(payload, key=lambda t: t[0])]
    gathered = [None] * world if rank == dst else None
    dist.gather_object(payload, gathered, dst=dst)
    if rank != dst:
        return None
    out = [None] * count
    for part in gathered:
        for i, s in part:
            out[i] = s
    return out
