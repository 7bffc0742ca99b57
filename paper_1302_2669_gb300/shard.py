"""Sharding of independent syndromes over ranks (one process per GPU).

Syndromes are independent and their randomness is keyed by the syndrome id,
so a batch splits across ranks with no exchange on the data path: rank r of
W decodes a contiguous id range, and only the results are combined at the
end (summed counters, the slowest rank's time, and an all-gather of the
per-syndrome decisions).  Works with any torch.distributed backend (NCCL on
GPUs, gloo on CPU).  `spawn_ranks` starts the ranks of one node.
"""
from __future__ import annotations

import socket
import subprocess
import sys


def free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def spawn_ranks(nproc: int, script: str, argv, port: int | None = None, env=None) -> int:
    """Runs `script argv` as `nproc` ranks of one node under
    torch.distributed.run (rendezvous on 127.0.0.1; every rank gets RANK,
    LOCAL_RANK, WORLD_SIZE and MASTER_*), waits for them and returns the
    launcher's exit code."""
    if nproc < 1:
        raise ValueError("nproc must be >= 1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={nproc}",
           "--master-addr", "127.0.0.1", "--master-port", str(port or free_port()), script, *map(str, argv)]
    return subprocess.call(cmd, env=env)


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


def all_gather_rows(t, device=None):
    """Every rank's tensor (same shape on all ranks) concatenated along the
    first axis in rank order, on every rank; with contiguous id ranges this
    is the job's result in id order."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1):
        return t
    t = t.contiguous() if device is None else t.to(device).contiguous()
    out = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    return torch.cat(out)
