"""Replicas across GPUs: the path shards by structure (independent
problems), so N processes each solve their own seeded structure with no
data-path collective; only the timing is combined.

One process per GPU (launched by torchrun); `torch.distributed` carries the
barrier around the timed region and the max-over-ranks reduction of the
elapsed time.  The functions here hold that host logic so that it can be
exercised with the gloo backend on CPU.
"""
from __future__ import annotations


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of the structure rank `rank` solves (weak scaling: one structure
    of the same recipe and size per rank)."""
    return base_seed + rank


def max_over_ranks(value: float, dist=None, device: str = "cpu") -> float:
    """The largest `value` over all ranks (the job's time is its slowest
    rank's); `value` itself when not distributed."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed, over the
    slowest rank's time."""
    return units_per_rank * world / seconds
