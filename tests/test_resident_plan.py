"""Host-only checks of the resident engine's slab plan (md_resident_plan, no
GPU): every replica's MD-cell rows are covered by its slabs exactly once, a
replica's slabs run on consecutive CTAs, slab capacities respect the list
index width, and the order in which CTAs run their slabs has no cycle of
waits (the slabs of a replica meet at barriers, so a cycle would deadlock)."""

import math

import numpy as np
import pytest

from paper_2101_01160_gb300 import inputs

SMEM = 232448 - 1024   # one CTA per SM of a GB300
GRID = 152


@pytest.fixture(scope="module")
def lib():
    from paper_2101_01160_gb300 import build, mdlg

    build.build()
    mdlg.load()
    return mdlg


def _ensemble(mdlg, R, seed, skin=0.4):
    Ns, phis, _ = inputs.ensemble_params(R, seed=seed)
    out = []
    for n, phi in zip(Ns, phis):
        L = inputs.box_length(int(n), float(phi))
        out.append(mdlg.make_params(int(n), L, precision=mdlg.MD_FP32_CELLOFF, W=4, lg_every=(400,),
                                    lx=(int(round(L)),), skin=skin))
    return out


def _check(mdlg, params, grid=GRID):
    jobs, start, span = mdlg.resident_plan(params, grid, SMEM)
    assert span > 0 and len(start) == grid + 1 and start[0] == 0
    by_rep = {}
    for c in range(grid):
        for j in jobs[start[c]:start[c + 1]]:
            rep, g, k, r0, r1, p_cap, h_cap, cta0 = (int(v) for v in j)
            assert cta0 + k == c                       # slab k runs on CTA cta0 + k
            assert p_cap + 2 * h_cap <= 1 << 14 and p_cap <= 8192
            by_rep.setdefault(rep, []).append((k, g, r0, r1, p_cap, h_cap))
    assert sorted(by_rep) == list(range(len(params)))
    for rep, sl in by_rep.items():
        p = params[rep]
        nc = int(math.floor(p.box_L / (p.rc + p.skin)))
        sl.sort()
        g = sl[0][1]
        assert [s[0] for s in sl] == list(range(g))
        assert sl[0][2] == 0 and sl[-1][3] == nc
        for a, b in zip(sl, sl[1:]):
            assert a[3] == b[2]                         # rows tile [0, nc)
        if g > 1:
            assert all(s[3] - s[2] >= 2 for s in sl)   # a slab's halo rows differ
            assert all(s[5] > 0 for s in sl)
        # room for the expected particles of the largest slab
        rows = max(s[3] - s[2] for s in sl)
        assert sl[0][4] >= p.n * rows / nc
    # no cycle of waits: order replicas by their position on each CTA
    succ = {r: set() for r in by_rep}
    for c in range(grid):
        reps = [int(j[0]) for j in jobs[start[c]:start[c + 1]]]
        for a, b in zip(reps, reps[1:]):
            succ[a].add(b)
    indeg = {r: 0 for r in succ}
    for a in succ:
        for b in succ[a]:
            indeg[b] += 1
    ready = [r for r in succ if indeg[r] == 0]
    seen = 0
    while ready:
        a = ready.pop()
        seen += 1
        for b in succ[a]:
            indeg[b] -= 1
            if indeg[b] == 0:
                ready.append(b)
    assert seen == len(succ)
    return jobs, start


def test_plan_of_the_bench_ensemble(lib):
    jobs, start = _check(lib, _ensemble(lib, 256, seed=7))
    # every CTA gets work


@pytest.mark.parametrize("R,seed", [(3, 1), (40, 2), (300, 3)])
def test_plan_of_other_ensembles(lib, R, seed):
    _check(lib, _ensemble(lib, R, seed=seed))


def test_plan_single_small_and_large_replicas(lib):
    for n, phi in ((2000, 0.05), (65536, 0.3), (65536, 0.02), (200_000, 0.1)):
        L = inputs.box_length(n, phi)
        _check(lib, [lib.make_params(n, L, precision=lib.MD_FP32_CELLOFF, lx=(int(L),), skin=0.4)], grid=GRID)


def test_plan_rejects_replica_without_slab(lib):
    # a replica far denser than any liquid cannot fit the list capacity of
    # one slab of two cell rows
    n = 400_000
    L = 100.0
    p = lib.make_params(n, L, precision=lib.MD_FP32_CELLOFF, lx=(100,), skin=0.4)
    with pytest.raises(lib.MDError):
        lib.resident_plan([p], GRID, SMEM)
