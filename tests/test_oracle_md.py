"""Pins of the oracle's Lennard-Jones force and velocity-Verlet dynamics (Sec. 4):
exact potential values, force = -grad of the potential by finite differences,
Newton's third law, cell list = all pairs, NVE energy error scaling as dt^2,
momentum conservation, time reversibility, the energy of a hand-made
configuration, and the ballistic ideal gas whose
measured equilibrium must equal the Gaussian one (Sec. 1) within sampling
error."""

import math

import numpy as np
import pytest
from scipy import stats

from paper_2101_01160_gb300 import inputs


def test_pair_potential_values(orc):
    vc = 4 * (2.5 ** -12 - 2.5 ** -6)
    assert abs(vc - (-0.016316891136)) < 1e-15
    v, fr = orc.lj_pair(1.0)
    assert abs(v - (0.0 - vc)) < 1e-15 and abs(fr - 24.0) < 1e-13
    rmin = 2 ** (1 / 6)
    v, fr = orc.lj_pair(rmin * rmin)
    assert abs(v - (-1.0 - vc)) < 1e-14 and abs(fr) < 1e-13
    v, fr = orc.lj_pair(2.5 * 2.5 * (1 - 1e-15))
    assert abs(v) < 1e-15 and fr < 0    # shifted energy vanishes at rc, force attractive


def _system(n, L, seed, min_sep=0.8):
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = rng.uniform(0, L, 2)
        ok = True
        for q in pts:
            d = p - q
            d -= L * np.round(d / L)
            if d @ d < min_sep ** 2:
                ok = False
                break
        if ok:
            pts.append(p)
    a = np.array(pts)
    return a[:, 0].copy(), a[:, 1].copy()


def test_force_is_minus_gradient(orc):
    L = 9.0
    x, y = _system(40, L, 1)
    fx, fy, pe, _ = orc.forces_brute(x, y, L)
    U = lambda xx, yy: orc.forces_brute(xx, yy, L)[2].sum()
    h = 1e-6
    for i in range(0, 40, 3):
        for arr, f in ((x, fx), (y, fy)):
            p = arr.copy(); p[i] += h
            m = arr.copy(); m[i] -= h
            if arr is x:
                d = -(U(p, y) - U(m, y)) / (2 * h)
            else:
                d = -(U(x, p) - U(x, m)) / (2 * h)
            assert abs(d - f[i]) < 1e-5 * max(1.0, abs(f[i])), (i, d, f[i])


def test_newton_third_law_and_cells(orc):
    for n, L in ((300, 30.0), (30, 7.6), (50, 8.0), (500, 60.0), (20, 6.0)):
        x, y = _system(n, L, n, min_sep=0.7)
        fx, fy, pe, fa = orc.forces_brute(x, y, L)
        assert abs(fx.sum()) < 1e-10 * max(1, np.abs(fx).sum())
        assert abs(fy.sum()) < 1e-10 * max(1, np.abs(fy).sum())
        cx, cy, cpe, cfa = orc.forces_cells(x, y, L)
        assert np.max(np.abs(cx - fx)) < 1e-12 * max(1, fa.max())
        assert np.max(np.abs(cy - fy)) < 1e-12 * max(1, fa.max())
        assert np.max(np.abs(cpe - pe)) < 1e-13
        if int(L // 2.5) >= 3:    # below 3 cells per edge the cell list is not used
            sub = np.arange(0, n, 7)
            sx, sy, _, _ = orc.forces_cells(x, y, L, subset=sub)
            assert np.array_equal(sx[sub], cx[sub])


def _energy_error(orc, dt, t_end=0.4):
    st = inputs.lattice_gas_state(256, inputs.box_length(256, 0.3), 2.0, seed=9)
    r = orc.md_run(st.x, st.y, st.vx, st.vy, st.L, dt, int(round(t_end / dt)), energy_log=True)
    E = r["elog"][:, 0] + r["elog"][:, 1]
    return np.max(np.abs(E - E[0])), r


def test_nve_energy_error_scales_as_dt_squared(orc):
    e1, r1 = _energy_error(orc, 2e-3)
    e2, _ = _energy_error(orc, 1e-3)
    ratio = e1 / e2
    assert 3.0 < ratio < 5.5, ratio
    P = r1["elog"][:, 2:]
    assert np.max(np.abs(P)) < 1e-11


def test_time_reversal(orc):
    st = inputs.lattice_gas_state(400, inputs.box_length(400, 0.0784), 20.0, seed=3)
    r = orc.md_run(st.x, st.y, st.vx, st.vy, st.L, 5e-4, 300)
    b = orc.md_run(r["x"], r["y"], -r["vx"], -r["vy"], st.L, 5e-4, 300)
    d = b["x"] - st.x
    d -= st.L * np.round(d / st.L)
    assert np.max(np.abs(d)) < 1e-9
    assert np.max(np.abs(-b["vx"] - st.vx)) < 1e-8


def test_ballistic_ideal_gas_is_gaussian(orc):
    """Non-interacting particles: displacement over dt_lg is v*dt_lg with
    v ~ N(0, T/m), so the measured equilibrium equals f^{eq,G} with
    a^2 = T dt_lg^2 / dx^2 (Sec. 1: the ballistic regime is a single
    Gaussian)."""
    n, L, T = 200_000, 400.0, 20.0
    st = inputs.ideal_gas_state(n, L, T, seed=21)
    dt, S, lx, W = 0.01, 10, 400, 4
    r = orc.md_run(st.x, st.y, st.vx, st.vy, L, dt, S, every=[S], lx=[lx], W=W, eps=0.0)
    hist = r["hist"][0, 0].astype(np.float64)
    assert hist.sum() + r["overflow"][0, 0] == n
    a2 = T * (S * dt) ** 2 / (L / lx) ** 2
    P = orc.feq_gaussian(a2, 0.0, 0.0, W)
    exp = n * P
    keep = exp > 20
    chi2 = float(np.sum((hist[keep] - exp[keep]) ** 2 / exp[keep]))
    dof = int(keep.sum()) - 1
    assert stats.chi2.sf(chi2, dof) > 1e-3, (chi2, dof)
    # second moment of the continuous displacement: mu2 = T dt_lg^2 per axis
    mu2 = r["mom"][0, 0] / (2 * n)
    assert abs(mu2 - T * (S * dt) ** 2) < 5 * T * (S * dt) ** 2 * math.sqrt(2 / (2 * n))


def test_small_system_runs_sampling(orc):
    st = inputs.lattice_gas_state(1024, inputs.box_length(1024, 0.0784), 20.0, seed=1)
    r = orc.md_run(st.x, st.y, st.vx, st.vy, st.L, 5e-4, 2000, n_equil=0, every=[400, 1000],
                   lx=[101, 50], W=4)
    assert list(r["nwin"]) == [5, 2]
    tot = r["hist"].sum(axis=2) + r["overflow"]
    assert np.array_equal(tot, np.array([[5 * 1024] * 2, [2 * 1024] * 2]))


def test_moments_independent_of_lattice_count(orc):
    """mu2, mu4 of Sec. 3(b) are moments of the continuous displacement: adding
    lattices must not change them, and they equal the directly computed
    moments of x(t+dt_lg) - x(t)."""
    n = 1024
    L = inputs.box_length(n, 0.0784)
    st = inputs.lattice_gas_state(n, L, 20.0, seed=3)
    a = orc.md_run(st.x, st.y, st.vx, st.vy, L, 5e-4, 400, every=[400], lx=[101], W=4)
    b = orc.md_run(st.x, st.y, st.vx, st.vy, L, 5e-4, 400, every=[400], lx=[101, 45, 14], W=4)
    assert np.array_equal(a["mom"], b["mom"])
    dx = a["x"] - st.x
    dy = a["y"] - st.y
    dx -= L * np.round(dx / L)
    dy -= L * np.round(dy / L)
    assert abs(a["mom"][0, 0] - np.sum(dx ** 2 + dy ** 2)) < 1e-9 * a["mom"][0, 0]
    assert abs(a["mom"][0, 1] - np.sum(dx ** 4 + dy ** 4)) < 1e-9 * a["mom"][0, 1]


@pytest.mark.parametrize("eps,sigma,mass", [(1.0, 1.0, 1.0), (1.5, 1.1, 2.0)])
def test_energy_of_a_hand_made_configuration(orc, eps, sigma, mass):
    """Energy, momentum and the shifted potential summed once per pair under
    the minimum image (Sec. 4), written out for four particles in a 10 x 10
    box: pairs (0,1) at r = 1.1, (0,2) at 1.5 across the x wrap and (0,3)
    at 2.4 are inside rc = 2.5; every other pair is beyond it."""
    L, rc = 10.0, 2.5
    x = np.array([1.0, 2.1, 9.5, 1.0])
    y = np.array([1.0, 1.0, 1.0, 3.4])
    vx = np.array([0.5, -1.0, 2.0, 0.0])
    vy = np.array([1.5, 0.25, -0.75, -2.0])

    def v_shift(r):
        return 4 * eps * ((sigma / r) ** 12 - (sigma / r) ** 6) - 4 * eps * ((sigma / rc) ** 12 - (sigma / rc) ** 6)

    ke = 0.5 * mass * float(np.sum(vx * vx + vy * vy))
    pe = v_shift(1.1) + v_shift(1.5) + v_shift(2.4)
    out = orc.energy(x, y, vx, vy, L, rc=rc, eps=eps, sigma=sigma, mass=mass)
    assert abs(out[0] - ke) <= 1e-14 * ke
    assert abs(out[1] - pe) <= 1e-12 * abs(pe)
    assert abs(out[2] - mass * vx.sum()) <= 1e-15 and abs(out[3] - mass * vy.sum()) <= 1e-15
