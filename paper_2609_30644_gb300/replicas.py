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


def assign(costs, world: int) -> list:
    """Whole problems to ranks (one GPU each): the largest estimated cost
    first, each to the rank with the least load so far (ties: the lower
    rank), so that loads differ by at most one problem's cost.  Returns, per
    rank, its problem indices in ascending order; every rank computing this
    from the same costs gets the same partition."""
    loads = [0.0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i)):
        r = min(range(world), key=lambda k: (loads[k], k))
        loads[r] += float(costs[i])
        out[r].append(i)
    return [sorted(o) for o in out]


def problem_cost(scene) -> float:
    """Planning cost estimate of a scene for assign(): robots and obstacles
    drive the validation work (robot pairs, link-obstacle tests)."""
    K = len(scene.robots)
    n_obs = len(scene.obs_spheres) + len(scene.obs_cuboids)
    links = sum(r.dof for r in scene.robots)
    return float(links * (n_obs + 1) + 49 * K * (K - 1) // 2)


def dispatch(dist, costs, solve, rank: int, world: int) -> list:
    """Runs solve(i) for this rank's problems (assign) and gathers every
    rank's results; returns the results of all problems in problem order on
    every rank (None for a problem nobody solved).  With dist None (one
    rank) everything runs here.  solve's result must be picklable."""
    mine = assign(costs, world)[rank] if world > 1 else list(range(len(costs)))
    local = {i: solve(i) for i in mine}
    if dist is None or world <= 1:
        parts = [local]
    else:
        parts = [None] * world
        dist.all_gather_object(parts, local)
    out = [None] * len(costs)
    for part in parts:
        for i, v in part.items():
            out[i] = v
    return out
