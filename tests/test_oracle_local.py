"""Pins of the oracle's local MDLG fields (Sec. 2): the occupation numbers
n_i(x, t) of Eq. (n_i) per lattice site and the lattice-gas collision
operator Xi_i of Eq. (mdlg_evolution).

- Eq. (n_i) written out as its indicator sum on tiny inputs: cell membership
  tested as an interval, x - v_i taken on the periodic lattice (a sign or
  arrival/departure mix-up fails it).
- Summed over the sites, n_i is the global displacement histogram of
  or_bin_celloff (pinned in test_oracle_binning.py); the overflow too.
- Summed over the classes (plus the overflow), n_i(x, t1) is the population
  of site x at t1, whatever t0 is.
- Mass conservation: sum_i Xi_i(x, t) = 0 at every site when no
  displacement leaves the window (both sides count the particles at x at t).
- Free streaming at a whole number of lattice sites per window has no
  collisions (Xi = 0); a particle moving half a site per window has the
  hand-counted Xi of a lattice collision.
"""

import numpy as np
import pytest

from paper_2101_01160_gb300 import inputs


def _pair(a, b):
    return dict(cell0=a["cell"], ox0=a["ox"], oy0=a["oy"], cell1=b["cell"], ox1=b["ox"], oy1=b["oy"])


def _snap(xs, ys, ncell, h):
    """Exact dyadic positions -> (cell, offset) snapshot in FP64."""
    cx = np.floor(np.asarray(xs) / h).astype(np.int64)
    cy = np.floor(np.asarray(ys) / h).astype(np.int64)
    return dict(cell=(cy * ncell + cx).astype(np.int32), ox=np.asarray(xs) - cx * h,
                oy=np.asarray(ys) - cy * h)


def _member(p, X, dxl):
    # indicator of lattice cell X as an interval test
    return X * dxl <= p < (X + 1) * dxl


@pytest.mark.parametrize("lx,W", [(5, 2), (7, 1), (6, 2)])
def test_indicator_sum_definition(orc, lx, W):
    ncell, h = 8, 1.25
    L = ncell * h
    dxl = L / lx
    rng = np.random.Generator(np.random.PCG64(lx * 10 + W))
    n = 40
    # dyadic positions (multiples of 1/64) so that membership is exact
    g = lambda: rng.integers(0, int(L * 64), n) / 64.0   # noqa: E731
    x0, y0, x1, y1 = g(), g(), g(), g()
    s = _pair(_snap(x0, y0, ncell, h), _snap(x1, y1, ncell, h))
    nf, ovf = orc.site_occupation(s, ncell, h, L, lx, W)
    side = 2 * W + 1
    ref = np.zeros_like(nf)
    for Y in range(lx):
        for X in range(lx):
            for vy in range(-W, W + 1):
                for vx in range(-W, W + 1):
                    Xs, Ys = (X - vx) % lx, (Y - vy) % lx
                    ref[(vy + W) * side + (vx + W), Y, X] = sum(
                        _member(x1[j], X, dxl) and _member(y1[j], Y, dxl)
                        and _member(x0[j], Xs, dxl) and _member(y0[j], Ys, dxl) for j in range(n))
    assert np.array_equal(nf, ref)
    # the rest of each site's arrivals leave the window: with lx <= 2W + 1 none
    pop1 = np.zeros((lx, lx), np.int64)
    for j in range(n):
        pop1[int(y1[j] // dxl), int(x1[j] // dxl)] += 1
    assert np.array_equal(nf.sum(axis=0) + ovf, pop1)
    if lx <= side:
        assert ovf.sum() == 0


@pytest.mark.parametrize("f64", [False, True])
@pytest.mark.parametrize("lx,W", [(101, 4), (37, 1), (64, 10)])
def test_sum_over_sites_is_the_global_histogram(orc, f64, lx, W):
    ncell, h = 33, 101.283 / 33
    L = ncell * h
    s = inputs.random_celloff_snapshots(5000, ncell, h, seed=lx + W, max_step=6.0, f64=f64,
                                        ties=300, lattice_dx=L / lx)
    nf, ovf = orc.site_occupation(s, ncell, h, L, lx, W)
    hist, ov, _ = orc.bin_celloff(s, ncell, h, L, lx, W)
    assert np.array_equal(nf.sum(axis=(1, 2)), hist)
    assert int(ovf.sum()) == ov


def test_class_sum_is_the_arrival_population(orc):
    ncell, h, lx, W = 16, 2.5, 20, 2
    L = ncell * h
    walk = inputs.random_celloff_walk(3000, ncell, h, seed=4, max_step=3.0, steps=2, f64=True)
    # the same t1 seen from two different t0: same per-site totals
    a, oa = orc.site_occupation(_pair(walk[0], walk[2]), ncell, h, L, lx, W)
    b, ob = orc.site_occupation(_pair(walk[1], walk[2]), ncell, h, L, lx, W)
    assert np.array_equal(a.sum(axis=0) + oa, b.sum(axis=0) + ob)
    # t0 = t1: everything stays, n_0(x) is the population of x
    c, oc = orc.site_occupation(_pair(walk[2], walk[2]), ncell, h, L, lx, W)
    side = 2 * W + 1
    zero = W * side + W
    assert oc.sum() == 0
    assert np.array_equal(np.delete(c, zero, axis=0), np.zeros_like(np.delete(c, zero, axis=0)))
    assert np.array_equal(c[zero], b.sum(axis=0) + ob)
    assert c[zero].sum() == 3000


@pytest.mark.parametrize("f64", [False, True])
def test_collision_conserves_mass_at_every_site(orc, f64):
    ncell, h, lx, W = 24, 2.75, 30, 3
    L = ncell * h
    walk = inputs.random_celloff_walk(20000, ncell, h, seed=9, max_step=4.0, steps=2, f64=f64)
    n1, o1 = orc.site_occupation(_pair(walk[0], walk[1]), ncell, h, L, lx, W)
    n2, o2 = orc.site_occupation(_pair(walk[1], walk[2]), ncell, h, L, lx, W)
    assert o1.sum() == 0 and o2.sum() == 0        # steps of at most 1.8 sites
    xi = orc.collision(n1, n2, W)
    assert np.array_equal(xi.sum(axis=0), np.zeros((lx, lx), np.int64))
    assert np.abs(xi).sum() > 0
    # the evolution equation read back: n_i(x + v_i, t + dt) = n_i(x, t) + Xi_i
    side = 2 * W + 1
    for vy in range(-W, W + 1):
        for vx in range(-W, W + 1):
            i = (vy + W) * side + (vx + W)
            assert np.array_equal(np.roll(n2[i], (-vy, -vx), axis=(0, 1)), n1[i] + xi[i])


def test_free_streaming_has_no_collisions(orc):
    ncell, h, lx, W = 8, 2.0, 8, 2
    L = ncell * h
    dxl = L / lx
    # one particle per class, starting at distinct site centres, moving a
    # whole number of sites per window
    v = [(vx, vy) for vy in range(-W, W + 1) for vx in range(-W, W + 1)]
    x0 = np.array([(k % lx + 0.5) * dxl for k in range(len(v))])
    y0 = np.array([(k // lx + 0.5) * dxl for k in range(len(v))])
    snaps = [_snap(np.mod(x0 + t * dxl * np.array([a for a, _ in v]), L),
                   np.mod(y0 + t * dxl * np.array([b for _, b in v]), L), ncell, h) for t in range(3)]
    n1, o1 = orc.site_occupation(_pair(snaps[0], snaps[1]), ncell, h, L, lx, W)
    n2, o2 = orc.site_occupation(_pair(snaps[1], snaps[2]), ncell, h, L, lx, W)
    assert o1.sum() == 0 and n1.sum() == len(v)
    assert np.array_equal(orc.collision(n1, n2, W), np.zeros_like(n1))


def test_half_site_velocity_collides(orc):
    ncell, h, lx, W = 8, 2.0, 8, 1
    L = ncell * h
    dxl = L / lx
    # x = 0.5, 1.0, 1.5 sites (cells 0 -> 1 -> 1): displacement (1,0) then (0,0)
    snaps = [_snap([f * dxl], [0.5 * dxl], ncell, h) for f in (0.5, 1.0, 1.5)]
    n1, _ = orc.site_occupation(_pair(snaps[0], snaps[1]), ncell, h, L, lx, W)
    n2, _ = orc.site_occupation(_pair(snaps[1], snaps[2]), ncell, h, L, lx, W)
    side = 2 * W + 1
    i10, i00 = W * side + (1 + W), W * side + W
    assert n1[i10, 0, 1] == 1 and n1.sum() == 1
    assert n2[i00, 0, 1] == 1 and n2.sum() == 1
    xi = orc.collision(n1, n2, W)
    # Xi_(1,0)(x=1) = n_(1,0)(x=2, t+dt) - n_(1,0)(x=1, t) = -1
    # Xi_(0,0)(x=1) = n_(0,0)(x=1, t+dt) - n_(0,0)(x=1, t) = +1
    expect = np.zeros_like(xi)
    expect[i10, 0, 1] = -1
    expect[i00, 0, 1] = 1
    assert np.array_equal(xi, expect)
