"""Frame sharding across ranks (one process per GPU).

Frames of an animation are independent problems: rank r renders frames
r * stride + k of the same scene, so the ranks never exchange data on the
rendering path (weak scaling). The only collective is the measurement's
max-over-ranks of the timed total.
"""
from __future__ import annotations

from typing import List

FRAME_STRIDE = 100000


def rank_frames(rank: int, world: int, count: int, start: int = 0) -> List[int]:
    """Frame indices rank `rank` of `world` renders: `count` consecutive frames
    from its own block, disjoint from every other rank's."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base = rank * FRAME_STRIDE + start
    return list(range(base, base + count))


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of `value` over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: int, max_seconds: float) -> float:
    """Whole-job throughput: units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / max_seconds
