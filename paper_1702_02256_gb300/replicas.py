"""Multi-GPU weak scaling by independent replicas.

Templates are independent (Eqs. iireq0, iireq1: every template's SNR depends
only on its own filters and the shared strain), so N GPUs run N independent
banks on the same strain with no collective on the data path. The only
cross-rank steps are host-side: a barrier around the timed region and the
maximum of the per-rank times, which makes the whole-job rate
(units of all ranks) / (slowest rank's time)."""
from __future__ import annotations

import os


def world():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s bank: distinct banks of the same shape per rank."""
    return base + 1000 * rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without dist)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world_size: int, seconds_max: float) -> float:
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    return world_size * units_per_rank / seconds_max
