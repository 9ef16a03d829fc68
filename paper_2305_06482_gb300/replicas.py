"""Replicas across ranks (one process per GPU, launched by torchrun).

A reconstruction of one volume does not shard without an image-sized all-reduce per adjoint, so
N ranks run N independent reconstructions, each of its own synthetic volume; nothing is
exchanged on the data path.  Only the timing is combined: the whole job made N x K
reconstructions in the time of the slowest rank (weak scaling).
"""
from __future__ import annotations

import torch


def replica_seed(base: int, rank: int) -> int:
    """Phantom seed of a rank's volume (distinct per rank, rank 0 keeps the base seed)."""
    return base + 17 * rank


def slowest_ms(ms_local: float, dist=None, device=None) -> float:
    """Max over ranks of a per-rank duration in ms (the local value when not distributed)."""
    if dist is None:
        return float(ms_local)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def seconds_per_recon(ms_slowest: float, steps: int, world: int) -> float:
    """Whole-job seconds per reconstruction: world x steps reconstructions in ms_slowest."""
    return ms_slowest / 1e3 / (steps * world)
