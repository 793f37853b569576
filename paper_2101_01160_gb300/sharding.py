"""Host logic of the replica-sharded multi-GPU run (one process per GPU).

Replicas are independent, so ranks share no data: rank r runs its own
seeded ensemble (seed offset r) and nothing is exchanged during the timed
region.  After it, one reduction gives the whole-job figures: the units
(particle-steps) summed over ranks and the timed region's maximum over
ranks, so the aggregate rate is sum(units) / max(time).
"""

from __future__ import annotations

import os


def world():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def seed_offset(rank: int) -> int:
    """Seed offset of rank's ensemble: distinct draws per rank."""
    return rank


def aggregate(dist, units: float, ms: float):
    """(sum of units over ranks, max of ms over ranks); dist is
    torch.distributed (initialised) or None for a single process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(units), float(ms)
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())
