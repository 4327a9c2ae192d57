"""Frame sharding over ranks (one process per GPU).

Frames are independent, so N GPUs decode N independent batches (weak scaling) with no
collective on the data path; collectives serve only the timing barrier and the maximum
of the per-rank times. Rank r's batch is the r-th block of frames of one global stream
of seeded batches, so the union over ranks is the same data whatever N is.
"""
from __future__ import annotations


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s batch (batch k of the global stream is seeded base_seed + k)."""
    return base_seed + rank


def frame_range(total: int, rank: int, world: int):
    """Contiguous [start, stop) share of `total` frames for `rank` (strong-scaling split)."""
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group (identity when alone)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
