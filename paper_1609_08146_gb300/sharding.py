"""Point sharding across GPUs (Sec. III.C.2's domain decomposition).

Observation points are independent, so each rank evaluates a contiguous
range of them with the full node table replicated; there is no exchange
during the computation.  Results stay sharded, or are gathered to one rank
by a host copy.  torch.distributed is used only for that gather and for
timing (barrier, max over ranks), never on the data path of a field sum.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int):
    """Contiguous [begin, end) of n items for `rank`; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def gather_points(local, n_total: int, dim: int, group=None, dst: int = 0):
    """Gather per-rank tensors sharded along `dim` (points) into one tensor on
    rank `dst` (host copy through the process group); other ranks get None.
    Shards may differ in size by one, as shard_range makes them."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    local = local.detach().cpu().contiguous()
    sizes = [shard_range(n_total, r, world) for r in range(world)]
    shape = list(local.shape)
    bufs = []
    for b, e in sizes:
        shape[dim] = e - b
        bufs.append(torch.empty(shape, dtype=local.dtype))
    if rank == dst:
        out = [None] * world
        out[dst] = local
        for r in range(world):
            if r != dst:
                dist.recv(bufs[r], src=r, group=group)
                out[r] = bufs[r]
        return torch.cat(out, dim=dim)
    dist.send(local, dst=dst, group=group)
    return None
