"""Sharding of independent syndromes over ranks (one process per GPU).

Syndromes are independent and their randomness is keyed by the syndrome id,
so a batch splits across ranks with no exchange on the data path: rank r of
W decodes a contiguous id range, and only the final counters (failures,
syndromes, elapsed time) are combined.  Works with any torch.distributed
backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations


def id_range(rank: int, world: int, n_total: int):
    """Contiguous share of ids 0..n_total-1 for `rank`: (first id, count)."""
    if not (0 <= rank < world) or n_total < 0:
        raise ValueError("bad rank/world/n_total")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def weak_id0(rank: int, n_per_rank: int) -> int:
    """First id of a rank when every rank decodes n_per_rank syndromes."""
    return rank * n_per_rank


def sum_counts(values, device=None):
    """Sums a list of integers over all ranks (all-reduce)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.int64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [int(v) for v in t.tolist()]


def max_value(x: float, device=None) -> float:
    """Maximum of a float over all ranks (the job's time is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
