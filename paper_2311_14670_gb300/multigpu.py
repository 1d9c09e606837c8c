"""Host-side logic of multi-GPU runs: one process per GPU, independent work per rank.

Transforms of different signals are independent, so N GPUs shard whole batches (weak scaling)
with no collective on the data path.  torch.distributed is used only to line the ranks up before
and after the timed region and to take the maximum of the per-rank times.
"""
from __future__ import annotations

import os


def world_info() -> tuple:
    """(world_size, rank, local_rank) from the torchrun environment (defaults: one process)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_items: int, world: int, rank: int) -> range:
    """Contiguous, balanced share of n_items for rank (sizes differ by at most one)."""
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's synthetic inputs: distinct per rank, reproducible."""
    return base * 1000 + rank


def max_over_ranks(values, device=None):
    """Elementwise maximum of a list of floats over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def weak_scaling_throughput(units_per_rank: int, world: int, ms_max: float, steps: int) -> float:
    """Whole-job units per second: every rank's units divided by the slowest rank's time."""
    return units_per_rank * world * steps / (ms_max * 1e-3)
