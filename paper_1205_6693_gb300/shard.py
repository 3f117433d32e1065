"""Sharding of independent units (graphs, requests) across ranks.

A batch of independent graphs is split into contiguous, near-equal ranges,
one per rank; each rank decomposes its own range with no collective on the
data path (truss numbers of disjoint graphs are independent, Definition 2).
Only the timing is combined, as the maximum over ranks.
"""
from __future__ import annotations


def shard_range(units: int, rank: int, world: int) -> tuple[int, int]:
    """Half-open range [begin, end) of the units owned by `rank`."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(units, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def max_over_ranks(value: float) -> float:
    """Maximum of `value` over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
