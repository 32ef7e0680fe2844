"""Work split over ranks (one process per GPU) and the job-level timing.

Layout decomposition shards without any data exchange: sub-graphs, and
whole layouts, are independent (the task parallelism of Sec. 1 / Sec. 3).
Each rank decomposes its own layout; the only collectives are a barrier and
two scalar reductions that turn per-rank timings into a job throughput
(segments summed over ranks, time = the slowest rank).
"""
from __future__ import annotations


def rank_seed(seed: int, rank: int) -> int:
    """Seed of the layout rank ``rank`` decomposes (rank 0 keeps the workload's seed)."""
    return seed + 1000 * rank


def aggregate(dist, segments: float, seconds: float, device) -> tuple[float, float]:
    """(segments over all ranks, max seconds over ranks) via two all-reduces."""
    import torch

    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    s = torch.tensor([float(segments)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(s.item()), float(t.item())
