"""Walker sharding across processes (one GPU each) and the one exchange step of
the parallel multicanonical estimator (Sec. 2.2, Fig. 2): every rank runs its
own independent walkers with the shared weights, the histograms are summed
over ranks once per iteration, and every rank then applies the same
deterministic Berg update, so no weight broadcast is needed.

Only the histogram sum crosses ranks; the sweep itself has no collective.
"""
from __future__ import annotations

import os

import torch


def world() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment (1 process if unset)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def walker_seed_base(rank: int, walkers_per_rank: int) -> int:
    """Walker keys of rank r are r * walkers_per_rank + 0 .. walkers_per_rank - 1 (disjoint streams)."""
    return rank * walkers_per_rank


def combine_histograms(hist: torch.Tensor) -> torch.Tensor:
    """Sum a histogram tensor over all ranks in place (no-op for one process)."""
    if torch.distributed.is_available() and torch.distributed.is_initialized() \
            and torch.distributed.get_world_size() > 1:
        torch.distributed.all_reduce(hist, op=torch.distributed.ReduceOp.SUM)
    return hist


def max_over_ranks(x: float, device) -> float:
    """Largest value of x over the ranks (the job's time is its slowest rank's)."""
    if torch.distributed.is_available() and torch.distributed.is_initialized() \
            and torch.distributed.get_world_size() > 1:
        t = torch.tensor([x], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())
    return x
