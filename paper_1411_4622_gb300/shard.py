"""Multi-GPU layout of a batched run: each rank anneals its own contiguous
range of slices with its own copy of the PILA; there is no collective on the
data path (slices are independent problems), only a barrier and a MAX
reduction of the step time, so the whole-job rate is weak-scaled."""
from __future__ import annotations


def slice_range(rank: int, per_rank: int) -> tuple[int, int]:
    """(first global slice index, count) of a rank."""
    return rank * per_rank, per_rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest of every rank's value (the step time of the slowest rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_rate(world: int, units_per_rank_step: int, ms_per_step: float) -> float:
    """Units processed by all ranks per second."""
    return world * units_per_rank_step / (ms_per_step / 1e3)
