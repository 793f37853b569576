"""Host-side helpers of bench.py (no GPU): the per-replica Verlet skin of
the bench ensemble and the algorithmic flop count it enters."""

import math
import os
import sys

import numpy as np
import pytest

pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from paper_2101_01160_gb300 import inputs  # noqa: E402


def test_skin_follows_the_thermal_speed():
    # proportional to sqrt(T) above the floor: every replica uses its
    # displacement bound (max |v| dt per step over half its skin) at the
    # same rate as the hottest one
    Ts = np.linspace(1.0, 20.0, 96)
    sk = np.array([bench.skin_of(T) for T in Ts])
    assert np.all(np.diff(sk) >= 0) and sk.min() >= bench.SKIN_MIN
    assert bench.skin_of(bench.SKIN_T) == pytest.approx(bench.SKIN_HOT)
    free = sk > bench.SKIN_MIN
    ratio = sk[free] / np.sqrt(Ts[free])
    assert np.allclose(ratio, bench.SKIN_HOT / math.sqrt(bench.SKIN_T), rtol=1e-12)
    assert bench.skin_of(1.0) == bench.SKIN_MIN
    assert "0.7 sqrt(T/20)" in bench.WORKLOAD


def test_flop_count_uses_each_replicas_skin():
    Ns, phis, Ts = inputs.ensemble_params(32, seed=7)
    ens = [(int(n), inputs.box_length(int(n), float(f)), float(f), float(t), None)
           for n, f, t in zip(Ns, phis, Ts)]
    per_rep = bench._flops_per_particle_step(ens)
    hot = bench._flops_per_particle_step(ens, skin=bench.SKIN_HOT)
    floor = bench._flops_per_particle_step(ens, skin=bench.SKIN_MIN)
    assert floor < per_rep < hot
    # written out: 5 flops per listed pair, 13 per pair within rc, 16 per particle
    num = sum(n * (5 * math.pi * (2.5 + bench.skin_of(T)) ** 2 * n / L ** 2
                   + 13 * math.pi * 2.5 ** 2 * n / L ** 2 + 16) for (n, L, _, T, _) in ens)
    assert per_rep == pytest.approx(num / sum(e[0] for e in ens), rel=1e-12)
    # all replicas at the skin's reference temperature: the uniform count
    same = [(n, L, f, bench.SKIN_T, None) for (n, L, f, _, _) in ens]
    assert bench._flops_per_particle_step(same) == pytest.approx(hot, rel=1e-12)
