"""Probe sharding across ranks.

The stochastic estimator is a sum over independent probes, and the paper's
parallel scheme splits the samples among processes with one reduction before
the trace.  Rank r evaluates the global probes r R .. r R + R - 1 by shifting
the seed of the probe rule (u_{l,i} from SplitMix64(seed + (l << 32) + i)), and
the per-rank energy and force estimates, each over R probes, are averaged: the
mean equals the estimate over all W R probes.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_seed(seed: int, rank: int, n_probes_per_rank: int) -> int:
    """Seed whose local probes 0..R-1 are the global probes rank R .. rank R + R - 1."""
    return (int(seed) + ((int(rank) * int(n_probes_per_rank)) << 32)) % (1 << 64)


def reduce_estimates(energy: torch.Tensor, forces: torch.Tensor | None = None, group=None) -> None:
    """In place: the mean over ranks of the energy (and forces) estimates."""
    world = dist.get_world_size(group)
    dist.all_reduce(energy, group=group)
    energy.div_(world)
    if forces is not None:
        dist.all_reduce(forces, group=group)
        forces.div_(world)
