"""Pins against the values the paper prints for its simulation setup
(Table 1 and Sec. 4, stored in tests/golden/table1_setup.txt with the
citation): the lattice-commensurability reading lx = round(L / dx), the
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
        # lx = round(L / dx) reproduces every printed lattice size but one
        if int(round(L / dx)) != int(lx) or abs(lx * dx - L) > 1e-6 * L:
            inconsistent.append((dx, int(lx)))
        # dt_lg = MD step x output frequency; total = iterations x dt_lg
        assert math.isclose(freq * setup["md_step"], dt_lg, rel_tol=0, abs_tol=5e-5)
        assert math.isclose(setup["iterations"] * dt_lg, total, rel_tol=0, abs_tol=0.05)
    # the garbled row: 180 x 5.5 = 990, not L (lx = round(L / dx) = 182 is taken)
    assert inconsistent == [(5.5, 180)]


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
