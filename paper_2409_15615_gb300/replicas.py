"""Multi-GPU bookkeeping for independent registration pairs.

Pairs are independent, so N GPUs run N replicas: each rank takes its own
share of the pairs (or its own pair seed), there is no collective on the data
path, and the only communication is a barrier around the timed region and a
max-reduction of the per-rank times.  Whole-job throughput is all ranks'
units divided by the slowest rank's time.
"""
from __future__ import annotations

import os


def dist_env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def shard(n_items: int, rank: int, world: int):
    """Contiguous, balanced share [lo, hi) of n_items for this rank."""
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def pair_seed(base: int, rank: int) -> int:
    """Seed of the synthetic pair a rank times (weak scaling: one pair each)."""
    return base + rank


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank float over the default process group (identity
    without one).  Uses a CPU tensor for gloo, a device tensor for nccl."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(units_per_rank: float, world: int, max_seconds: float) -> float:
    """All ranks' units per second, timed by the slowest rank."""
    return world * units_per_rank / max_seconds
