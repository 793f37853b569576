"""Host-side analysis helpers of the non-equilibrium run (no GPU): the
sine/cosine/constant fit that reads the lattice-velocity and momentum-flux
profiles off the ensemble fields."""

import math

import numpy as np

from paper_2101_01160_gb300 import nonequilibrium


def test_fit_sine_recovers_the_profile():
    lx = 41
    k = 2.0 * math.pi / lx
    yc = np.arange(lx) + 0.5
    prof = 0.2279 * np.sin(k * yc) - 0.0089 * np.cos(k * yc) + 0.0011
    coef = nonequilibrium._fit_sine(prof, k, yc)
    assert np.allclose(coef, [0.2279, -0.0089, 0.0011], atol=1e-14)


def test_fit_sine_is_blind_to_other_wavelengths():
    # a second harmonic and a noise-free offset do not leak into the first
    # harmonic's coefficients (the rows span whole periods)
    lx = 40
    k = 2.0 * math.pi / lx
    yc = np.arange(lx) + 0.5
    prof = 0.1 * np.sin(k * yc) + 0.05 * np.sin(2 * k * yc) + 0.03 * np.cos(3 * k * yc)
    s, c, m = nonequilibrium._fit_sine(prof, k, yc)
    assert abs(s - 0.1) < 1e-14 and abs(c) < 1e-14 and abs(m) < 1e-14
