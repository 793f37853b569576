"""Pins against the values the paper prints for its simulation setup
(Table 1 and Sec. 4, stored in tests/golden/table1_setup.txt with the
citation): the lattice-commensurability check lx dx = L, the
relation between MD output frequency, MD step and coarse-grained step, the
area fraction of the standard system, and the statement that at the printed
a^2 ~ 0.1611 nearly every particle moves at most one lattice site per axis
(a D2Q9 lattice), evaluated with the oracle's Gaussian equilibrium."""

import math
import os
from fractions import Fraction

import numpy as np

from paper_2101_01160_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def _load():
    setup, rows = {}, []
    for line in open(os.path.join(HERE, "golden", "table1_setup.txt")):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        f = line.split()
        if len(f) == 2:
            setup[f[0]] = float(f[1])
        else:
            rows.append([float(Fraction(v)) for v in f])
    return setup, np.array(rows)


def test_table1_lattice_and_time_relations():
    setup, rows = _load()
    L = setup["L"]
    inconsistent = []
    for dt_lg, dx, lx, freq, total in rows:
        # lx dx = L holds for every printed row but one
        if int(round(L / dx)) != int(lx) or abs(lx * dx - L) > 1e-6 * L:
            inconsistent.append((dx, int(lx)))
        # dt_lg = MD step x output frequency; total = iterations x dt_lg
        assert math.isclose(freq * setup["md_step"], dt_lg, rel_tol=0, abs_tol=5e-5)
        assert math.isclose(setup["iterations"] * dt_lg, total, rel_tol=0, abs_tol=0.05)
    # the garbled row: 180 x 5.5 = 990, not L.  The reproduction takes lx = 180
    # (dx = L / 180 = 5.5(5), printed truncated): at dx = 5.5 the a^2 its own
    # MD measures would be 2% above the table's 0.1611, at L / 180 it is not.
    assert inconsistent == [(5.5, 180)]


def test_reproduction_rows_follow_the_table():
    from paper_2101_01160_gb300 import replicate

    setup, rows = _load()
    assert len(replicate.TABLE1) == len(rows)
    assert replicate.N == setup["N"] and replicate.L == setup["L"]
    assert replicate.A2_TABLE == setup["a2"]
    for (dt_lg, lx), row in zip(replicate.TABLE1, rows):
        assert dt_lg == row[0] and lx == int(row[2])


def test_d2q25_symmetric_sets():
    from paper_2101_01160_gb300 import replicate

    # the six sets partition the 25 nodes |vx|, |vy| <= 2 with sizes 1, 4, 4, 4, 8, 4
    W = 4
    side = 2 * W + 1
    sizes = []
    for k in range(len(replicate.SETS)):
        # the indicator of set k has mean 1 on set k and 0 on the others
        Q = np.zeros((side, side))
        for vy in range(-2, 3):
            for vx in range(-2, 3):
                if sorted((abs(vx), abs(vy))) == list(replicate.SETS[k]):
                    Q[vy + W, vx + W] = 1.0
        sizes.append(int(Q.sum()))
        assert replicate.set_means(Q.ravel(), W)[k] == 1.0
        assert np.all(np.delete(replicate.set_means(Q.ravel(), W), k) == 0.0)
    assert sizes == [1, 4, 4, 4, 8, 4]
    # the set means of a distribution weighted by set size sum to its total over D2Q25
    rng = np.random.Generator(np.random.PCG64(5))
    P = rng.random(side * side)
    m = replicate.set_means(P, W)
    tot = P.reshape(side, side)[W - 2:W + 3, W - 2:W + 3].sum()
    assert abs(float(np.dot(m, sizes)) - tot) < 1e-12


def test_area_fraction_of_the_standard_system():
    setup, _ = _load()
    phi = setup["N"] * math.pi / 4.0 / setup["L"] ** 2
    # the printed 0.078387 differs from N pi / (4 L^2) = 0.078427 by 5e-4 relative
    assert abs(phi - 0.078427) < 5e-7
    assert abs(phi - setup["phi"]) / phi < 1e-3
    # the box length the workloads derive from (N, phi) recovers L to the same accuracy
    assert abs(inputs.box_length(int(setup["N"]), setup["phi"]) - setup["L"]) / setup["L"] < 1e-3


def test_printed_a2_gives_a_d2q9_lattice(orc):
    setup, _ = _load()
    P = np.asarray(orc.feq_gaussian(setup["a2"], 0.0, 0.0, 4)).reshape(9, 9)
    d2q9 = P[3:6, 3:6].sum()
    assert d2q9 > 0.99                     # "most particles travel up to one lattice space"
    assert abs(P.sum() - 1.0) < 1e-12
