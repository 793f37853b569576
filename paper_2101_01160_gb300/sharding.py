"""Host logic of the replica-sharded multi-GPU run (one process per GPU).

Replicas are independent, so ranks share no data: rank r runs its own
seeded ensemble (seed offset r) and nothing is exchanged during the timed
region.  After it, one reduction gives the whole-job figures: the units
(particle-steps) summed over ranks and the timed region's maximum over
ranks, so the aggregate rate is sum(units) / max(time).

The one exchange of the method itself is at the end of a run whose ranks
sample the same state point: the measured equilibrium of all ranks together
(Eq. theory_feq over the union of their windows) needs the integer
histograms, overflow counts, particle-window totals and moment sums summed
over ranks; combine_measurements does that with one all-reduce.
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


def combine_measurements(dist, hist, overflow, samples, mom):
    """Sums one state point's measurements over ranks: hist (int64 counts per
    displacement class), overflow and samples (particle-windows) as exact
    integers, mom (sum of delta^2, sum of delta^4) in FP64 in rank order.
    Returns (hist, overflow, samples, mom, P, mu2, mu4) of the whole job, P =
    hist / samples (the measured f_eq per particle, Eq. theory_feq) and mu_k =
    mom_k / (2 samples) (both axes).  dist is torch.distributed (initialised)
    or None for a single process."""
    import numpy as np

    hist = np.asarray(hist, np.int64).copy()
    mom = np.asarray(mom, np.float64).copy()
    overflow, samples = int(overflow), int(samples)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        import torch

        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        ints = torch.tensor(np.concatenate([hist, [overflow, samples]]), dtype=torch.int64, device=dev)
        dist.all_reduce(ints, op=dist.ReduceOp.SUM)
        # FP64 sums in rank order (all_gather), so every rank gets the same bits
        parts = [torch.zeros(2, dtype=torch.float64, device=dev) for _ in range(dist.get_world_size())]
        dist.all_gather(parts, torch.tensor(mom, dtype=torch.float64, device=dev))
        v = ints.cpu().numpy()
        hist, overflow, samples = v[:-2], int(v[-2]), int(v[-1])
        mom = np.zeros(2)
        for t in parts:
            mom = mom + t.cpu().numpy()
    P = hist / float(samples) if samples else np.zeros(len(hist))
    mu2 = mom[0] / (2.0 * samples) if samples else 0.0
    mu4 = mom[1] / (2.0 * samples) if samples else 0.0
    return hist, overflow, samples, mom, P, mu2, mu4
