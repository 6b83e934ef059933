"""Multi-GPU bookkeeping for the benchmark: one process per GPU, each rank
evaluating its own shard of independent stacks (weak scaling: per-GPU work is
fixed), with no collective on the data path.  The only communication is the
barrier around the timed region and the max-over-ranks of the step time.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def barrier(device=None):
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
    if device is not None and torch.cuda.is_available():
        torch.cuda.synchronize(device)


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the whole-job step time)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: int, ms_per_rank: float, world: int, device=None) -> tuple:
    """(whole-job units per second, max step ms): units of all ranks over the
    slowest rank's time."""
    ms = max_over_ranks(ms_per_rank, device)
    return units_per_rank * world / (ms * 1e-3), ms
