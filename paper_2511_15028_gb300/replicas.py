"""Data-parallel replicas over several GPUs (one process per GPU).

Rays are independent, so every rank keeps its own copy of the BVH and traces a
contiguous shard of the rays; the hits are gathered on every rank (the only
exchange of the forward pass). The backward pass produces per-rank partial
sums of dL/dvertex that are added with one all-reduce; dL/dray stays sharded.

These helpers only move tensors: the tracing itself is the caller's
scion_trace_* call on its shard.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) of n items for `rank` of `world` (sizes differ
    by at most one, earlier ranks take the larger shares)."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def gather_shards(local, n_total: int, group=None):
    """All-gather per-rank shards (split by shard_range along dim 0) back into
    the full [n_total, ...] tensor on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    sizes = [shard_range(n_total, r, world) for r in range(world)]
    width = max(e - b for b, e in sizes)
    padded = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    padded[: local.shape[0]] = local
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    return torch.cat([p[: e - b] for p, (b, e) in zip(parts, sizes)], dim=0)


def allreduce_vertex_grads(grad_verts, group=None):
    """Sum the per-rank partial dL/dvertex in place (one all-reduce)."""
    import torch.distributed as dist
    dist.all_reduce(grad_verts, op=dist.ReduceOp.SUM, group=group)
    return grad_verts


def max_over_ranks(value: float, device="cpu", group=None) -> float:
    """Largest value over all ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
