"""Multi-GPU helpers of the benchmark: the path shards by solution interval.

Solution intervals are independent (Algorithm 1 loops over them), so ranks
share no data: under weak scaling every rank solves its own batch of
intervals (its own seed); under a fixed total every rank takes a contiguous
share of the intervals.  The only collectives are the benchmark's barrier
and the max over ranks of the timed region (torch.distributed, NCCL on GPUs,
gloo in the CPU tests).
"""
from __future__ import annotations

import os


def rank_info():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of a rank's own batch under weak scaling."""
    return int(base_seed) + int(rank)


def shard_intervals(n_intervals: int, world_size: int, rank: int):
    """Contiguous [begin, end) share of n_intervals for `rank` (sizes differ by at most one)."""
    q, r = divmod(int(n_intervals), int(world_size))
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def max_over_ranks(value: float, device="cpu") -> float:
    """The largest `value` over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
