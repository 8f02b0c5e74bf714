"""Multi-GPU runs of the operators are replicas: one process per GPU, each on its own independent
volumes, with no collective on the data path (every time step couples all voxels of a volume through
its spectrum, and a volume fits one GPU, so nothing is sharded).  Only the timing crosses ranks: the
job's time is the slowest rank's, and its throughput is the units all ranks processed over that time.
"""
from __future__ import annotations


def volume_seeds(rank: int, batch: int, stride: int = 100) -> list:
    """Phantom seed offsets of one rank's batch: disjoint across ranks for batch <= stride."""
    if batch > stride:
        raise ValueError("batch larger than the per-rank seed stride")
    return [stride * rank + b for b in range(batch)]


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return units_per_rank * world / seconds_max
