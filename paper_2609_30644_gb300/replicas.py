"""Replica-parallel execution over the GPUs of one node.

The hot path has no exchange step: edge batches, query batches and planning
problems are independent units, so every rank works on its own share and only
timing is combined (a barrier and a max over ranks).  Ranks come from the
torch.distributed.run environment (RANK, WORLD_SIZE, LOCAL_RANK, MASTER_*).
"""
from __future__ import annotations

import os
from typing import Optional


def env() -> tuple:
    """(rank, world_size, local_rank) from the launcher environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_units: int, rank: int, world: int) -> range:
    """Contiguous block of unit indices for this rank; blocks differ in size by
    at most one and together cover 0..n_units-1 exactly once."""
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def init(backend: str, device=None):
    """Joins the process group when more than one rank runs; returns the
    torch.distributed module or None for a single rank."""
    rank, world, _ = env()
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        kw = {"device_id": device} if device is not None and backend == "nccl" else {}
        dist.init_process_group(backend, **kw)
    return dist


def max_over_ranks(dist, value: float, device: Optional[object] = None) -> float:
    """Largest value over all ranks (the value itself for a single rank)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist) -> None:
    if dist is not None:
        dist.barrier()
