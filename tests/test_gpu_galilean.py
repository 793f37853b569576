"""Galilean-shifted equilibria (Eqs. feq_gaussian and p_wsg_one with a mean
velocity u, Sec. 3): MD of a dilute LJ gas (phi = 0.0784, T = 20) with a
uniform drift u = (2, 0) sigma/tau, sampled every Delta t = 1 on a lattice of
spacing ~4 sigma, so that the shift u Delta t / Delta x is about half a
lattice site.

The binning accumulates raw moments of the displacement, which include the
drift c = u_x Delta t on the x axis; with the thermal part symmetric, the
centred moments pooled over both axes follow exactly:
    var = mu2 - c^2 / 2,   mu4_c = mu4 - 3 c^2 var - c^4 / 2.
Checks: the measured mean lattice displacement equals the imposed shift
within sampling error; the shifted Gaussian at a^2 = var / Delta x^2 fits the
measured distribution far better than the unshifted one; the shifted WSG at
the centred moments fits better than the shifted Gaussian (as at u = 0).
"""

import math

import numpy as np
import pytest

from paper_2101_01160_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_drifting_gas_follows_shifted_equilibria(mdlg, orc):
    n, phi, T, ux = 65536, 0.0784, 20.0, 2.0
    every, dt, W = 2000, 5e-4, 4
    L = inputs.box_length(n, phi)
    st = inputs.lattice_gas_state(n, L, T, seed=31)
    lx = int(round(L / 4.0))
    p = mdlg.make_params(n, L, dt=dt, precision=mdlg.MD_FP32_CELLOFF, W=W, n_equil=4000,
                         lg_every=(every,), lx=(lx,))
    s = mdlg.System(p, st.x, st.y, st.vx + ux, st.vy)
    s.step(4000 + 10 * every)
    P, se, stats = s.feq_measured(0, 0, 0, symmetrize=False)
    s.close()
    dx = stats.dx_eff
    side = 2 * W + 1
    v = np.arange(side) - W
    Pm = P.reshape(side, side)                         # [vy][vx]
    assert stats.n_overflow < 1e-4 * stats.n_samples

    # mean lattice displacement = imposed shift (lattice units)
    u_lat = ux * every * dt / dx
    mean_x = float((Pm.sum(axis=0) * v).sum())
    mean_y = float((Pm.sum(axis=1) * v).sum())
    sigma_mean = math.sqrt(stats.mu2 / dx ** 2 / stats.n_samples) * 10.0   # windows are correlated
    assert abs(mean_x - u_lat) < 5 * sigma_mean + 2e-3, (mean_x, u_lat)
    assert abs(mean_y) < 5 * sigma_mean + 2e-3, mean_y

    # centred moments and the shifted equilibria
    c = ux * every * dt
    var = stats.mu2 - c * c / 2.0
    mu4c = stats.mu4 - 3.0 * c * c * var - c ** 4 / 2.0
    a2 = var / dx ** 2
    assert 3.0 < mu4c / var ** 2 < 3.75
    lam = float(mdlg.wsg_lambda(var, mu4c)[0].item())
    g_u = mdlg.feq_gaussian(a2, u_lat, 0.0, W).cpu().numpy()
    g_0 = mdlg.feq_gaussian(a2, 0.0, 0.0, W).cpu().numpy()
    w_u = mdlg.feq_wsg(a2, lam, u_lat, 0.0, W).cpu().numpy()
    # the analytic side against the oracle at this shift
    assert np.max(np.abs(g_u - orc.feq_gaussian(a2, u_lat, 0.0, W))) < 1e-12
    assert np.max(np.abs(w_u - orc.feq_wsg(a2, lam, u_lat, 0.0, W))) < 1e-12
    err_u = np.max(np.abs(P - g_u))
    err_0 = np.max(np.abs(P - g_0))
    assert err_u < 0.25 * err_0, (err_u, err_0)
    Pn = P / P.sum()
    assert orc.kl(Pn, w_u) < orc.kl(Pn, g_u), (orc.kl(Pn, w_u), orc.kl(Pn, g_u))
