"""Pins of the oracle's MDLG binning (Eq. n_i summed over the lattice, Sec. 2):
hand-counted snapshots with periodic wraps and boundary ties, exact mass
conservation, translation invariance by whole lattice cells, and the
(cell, offset) encoding decoding to the same positions."""

import numpy as np

from paper_2101_01160_gb300 import inputs


def _bin_index(ddx, ddy, W):
    return (ddy + W) * (2 * W + 1) + (ddx + W)


def test_hand_counted_snapshot(orc):
    L, lx, W = 10.0, 10, 2           # lattice spacing 1
    x0 = [0.5, 9.9, 1.0, 3.2, 5.5, 0.99, 4.0, 7.5]
    y0 = [0.5, 0.5, 2.0, 9.95, 5.5, 0.5, 4.0, 7.5]
    x1 = [1.5, 0.1, 0.999999, 3.2, 9.5, 1.0, 2.0, 7.5]
    y1 = [0.5, 9.9, 2.0, 0.05, 5.5, 0.5, 6.0, 7.5]
    # particle-by-particle (dx, dy) in lattice cells:
    #  0: cell 0 -> 1                         (+1, 0)
    #  1: x 9 -> 0 wraps forward, y 0 -> 9    (+1, -1)
    #  2: x exactly on line 1 -> cell 0       (-1, 0)   tie goes to the upper cell
    #  3: y 9 -> 0 wraps                      (0, +1)
    #  4: x 5 -> 9: |4| > W                   overflow
    #  5: x 0.99 (cell 0) -> 1.0 (cell 1)     (+1, 0)
    #  6: (4,4) -> (2,6)                      (-2, +2)
    #  7: no motion                           (0, 0)
    expect = np.zeros((2 * W + 1) ** 2, np.int64)
    for d in [(1, 0), (1, -1), (-1, 0), (0, 1), (1, 0), (-2, 2), (0, 0)]:
        expect[_bin_index(*d, W)] += 1
    hist, ovf, mom = orc.bin_xy(x0, y0, x1, y1, L, lx, W)
    assert ovf == 1
    assert np.array_equal(hist, expect)
    # continuous displacements, nearest image, both axes
    ex = np.array([1.0, 0.2, -1e-6, 0.0, 4.0, 0.01, -2.0, 0.0])
    ey = np.array([0.0, -0.6, 0.0, 0.1, 0.0, 0.0, 2.0, 0.0])
    assert abs(mom[0] - np.sum(ex ** 2 + ey ** 2)) < 1e-12
    assert abs(mom[1] - np.sum(ex ** 4 + ey ** 4)) < 1e-12


def test_odd_lattice_and_coarse_spacing(orc):
    # lx = 5 on L = 10: spacing 2; displacement of 3 cells wraps to -2
    L, lx, W = 10.0, 5, 2
    hist, ovf, _ = orc.bin_xy([0.5], [0.5], [6.5], [0.5], L, lx, W)
    assert ovf == 0 and hist[_bin_index(-2, 0, W)] == 1
    hist, ovf, _ = orc.bin_xy([0.5], [0.5], [4.5], [0.5], L, lx, W)
    assert hist[_bin_index(2, 0, W)] == 1
    # non-canonical positions (slightly outside [0, L)) map periodically
    hist, ovf, _ = orc.bin_xy([-0.5], [10.5], [0.5], [0.5], L, lx, W)
    assert hist[_bin_index(1, 0, W)] == 1


def test_mass_conservation_and_translation(orc):
    rng = np.random.default_rng(3)
    n, L = 20000, 101.283
    for lx, W in ((101, 4), (50, 2), (203, 4)):
        x0 = rng.uniform(0, L, n)
        y0 = rng.uniform(0, L, n)
        x1 = x0 + rng.normal(0, 1.5, n)
        y1 = y0 + rng.normal(0, 1.5, n)
        hist, ovf, mom = orc.bin_xy(x0, y0, x1, y1, L, lx, W)
        assert hist.sum() + ovf == n
        assert ovf > 0
        # shifting everything by whole lattice cells changes no count
        s = 7 * (L / lx)
        h2, o2, _ = orc.bin_xy(x0 + s, y0 - s, x1 + s, y1 - s, L, lx, W)
        # a shift can flip a point lying within rounding of a line; allow none here
        assert np.array_equal(h2, hist) or np.abs(h2 - hist).sum() <= 2


def test_zero_displacement_all_central(orc):
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 50, 1000)
    y = rng.uniform(0, 50, 1000)
    hist, ovf, mom = orc.bin_xy(x, y, x, y, 50.0, 37, 3)
    assert ovf == 0 and hist[_bin_index(0, 0, 3)] == 1000 and mom[0] == 0.0


def test_celloff_encoding_decodes_to_positions(orc):
    for f64 in (False, True):
        ncell, h = 33, 101.283 / 33
        s = inputs.random_celloff_snapshots(5000, ncell, h, seed=11, max_step=2.0, f64=f64,
                                            ties=200, lattice_dx=101.283 / 101)
        L = ncell * h
        hist, ovf, mom = orc.bin_celloff(s, ncell, h, L, 101, 4)
        cx0, cy0 = s["cell0"] % ncell, s["cell0"] // ncell
        cx1, cy1 = s["cell1"] % ncell, s["cell1"] // ncell
        X0 = cx0.astype(np.float64) * h + s["ox0"].astype(np.float64)
        Y0 = cy0.astype(np.float64) * h + s["oy0"].astype(np.float64)
        X1 = cx1.astype(np.float64) * h + s["ox1"].astype(np.float64)
        Y1 = cy1.astype(np.float64) * h + s["oy1"].astype(np.float64)
        h2, o2, m2 = orc.bin_xy(X0, Y0, X1, Y1, L, 101, 4)
        assert np.array_equal(hist, h2) and ovf == o2
        assert np.allclose(mom, m2, rtol=1e-12)
        assert hist.sum() + ovf == 5000
