"""Source sharding across processes (one GPU each).

Rays are independent, so the forward trace shards by source with no
collective: rank r traces the contiguous source range source_range(n, r, W)
and writes its own output rows.  The adjoint's per-leaf gradient is the only
quantity that needs a reduction: the per-rank partial gradients are summed
with one all-reduce.
"""
from __future__ import annotations


def source_range(n_src: int, rank: int, world: int):
    """Contiguous [s0, s1) of rank in a near-even split (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world or n_src < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_src, world)
    s0 = rank * base + min(rank, extra)
    return s0, s0 + base + (1 if rank < extra else 0)


def sharded_gradient(n_src: int, local_adjoint, group=None):
    """Sum over ranks of local_adjoint(s0, s1), the gradient contributed by this
    rank's sources; returns the full gradient on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    s0, s1 = source_range(n_src, rank, world)
    g = local_adjoint(s0, s1)
    if world > 1:
        dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return g
