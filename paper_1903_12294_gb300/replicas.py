"""Replica runs across ranks (one process per GPU): rank layout from the launcher's environment
and the reductions the measurement needs. Each rank holds the whole dataset and runs the same
work on its own GPU; there is no exchange on the data path (weak scaling)."""
from __future__ import annotations

import os


def layout():
    """(world, rank, local_rank) from the torchrun environment (1, 0, 0 when absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest value of x over all ranks (every rank gets it)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_throughput(units_per_rank: float, ms_max: float, world: int) -> float:
    """Whole-job throughput (units per second): every rank's units over the slowest rank's
    time."""
    return world * units_per_rank / (ms_max * 1e-3)
