"""Independent replicas across ranks (one process per GPU).

The lattice update has no exchange step between independent lattices, so N
GPUs run N independent lattices; the only communication is a barrier around
the timed region and the maximum of the per-rank times (gloo, host memory).
Launched by torchrun, which sets RANK, WORLD_SIZE, LOCAL_RANK and MASTER_*.
"""
from __future__ import annotations

import os


def ranks():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("gloo")


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def aggregate_rate(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (weak scaling: each rank has the same amount of work)."""
    return world * units_per_rank / seconds_max
