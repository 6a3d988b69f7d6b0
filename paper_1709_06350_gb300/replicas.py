"""Replica bookkeeping for multi-GPU runs (one process per GPU, torchrun).

Realisations are independent, so N GPUs run N replicas of the single-GPU
reconstruction with no collective in the data path; the only communication
is timing: a barrier around the timed region and the maximum elapsed time
over ranks.  Works with any torch.distributed backend (NCCL on GPUs, gloo in
the CPU tests).
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of this rank's realisation: distinct per rank, rank 0 keeps the base."""
    return base_seed + 7919 * rank


def barrier(dist=None) -> None:
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The slowest rank's value (the job's wall time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world_size: int, seconds_max: float) -> float:
    """Units processed by all ranks per second of the slowest rank (weak scaling)."""
    return units_per_rank * world_size / seconds_max
