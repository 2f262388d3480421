"""Counting one graph across several processes / GPUs (host-side exchange).

Every rank runs the whole levelling and row building and its share of the
intersection tasks (tc_count_shard); the exact total is the sum of the
partial counts -- one 8-byte all-reduce, the only exchange of the method.
Timing helpers take the maximum over ranks, as a job ends with its slowest
rank.
"""
from __future__ import annotations


def sum_partials(partial: int, group=None) -> int:
    """All-reduce SUM of one uint64 partial count (int64 on the wire; counts < 2^63)."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([partial], dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return int(t.item())


def max_over_ranks(value: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def count_sharded(ctx, g, group=None) -> int:
    """Exact T of g counted by all ranks of the process group together."""
    import torch.distributed as dist
    from . import tc_count_shard
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    partial, _ = tc_count_shard(ctx, g, rank, world)
    return sum_partials(partial, group)
