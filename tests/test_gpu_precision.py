"""Precision study at scale: one N = 4,194,304 state (phi = 0.0784,
L = 6482.12 sigma, T = 20, dt = 5e-4) advanced 2,000 steps in plain FP64 and
in the FP32 cell-index + offset encoding.

* forces: the subset is the particles of the central 136 x 136 MD cells
  (about 16,600); the oracle computes their FP64 forces from each system's
  raw state (cell index + offset) rewritten in local coordinates
  (cell - corner) * h + offset around that window with a one-cell halo
  (h >= rc + skin, and no particle has moved more than skin/2 since the last
  rebuild), in an open box wide enough that no pair wraps.  The bar is the
  one of the small tests, |F - F_oracle| <= tol * sum_j |F_ij| with tol 1e-12
  (FP64) and 1e-5 (FP32), plus the effect of the oracle's own input rounding:
  each local coordinate carries up to u = ulp(box) / 2, so a pair vector is off
  by up to 2 sqrt(2) u and the pair force F(r) r_hat by up to
  (|F'(r)| + |F(r)| / r) 2 sqrt(2) u; in FP32 the kernel forms each pair
  vector component as dcell * h + (off_j - off_i), two roundings of
  magnitude <= 2h at unit roundoff 2^-24, which adds 2 sqrt(2) 2^-24 2h to
  that displacement bound (near the zero of the LJ force, r ~ 1.12, these
  terms dominate sum_j |F_ij|);
* energy: relative drift of the total (shifted) energy over the 2,000 steps,
  with the bars of the small conservation test (5e-5 FP64, 1e-3 FP32);
* f_eq: the measured distributions of the two encodings over the same five
  sampling windows (every 400 steps on a lattice of spacing ~1 sigma) agree
  class by class within 6 multinomial standard errors of a difference.
"""

import numpy as np
import pytest

from paper_2101_01160_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, PHI, T, STEPS, EVERY = 4_194_304, 0.0784, 20.0, 2000, 400


def _forces_vs_oracle(s, orc, tol, fp32, wc=136):
    info = s.rep_info(0)
    nc, h = int(info.ncell), float(info.h)
    cell, ox, oy = s.get_raw()
    cell = cell.cpu().numpy().astype(np.int64)
    ox = ox.cpu().numpy().astype(np.float64)
    oy = oy.cpu().numpy().astype(np.float64)
    cx, cy = cell % nc, cell // nc
    c0 = nc // 2 - wc // 2
    win = (cx >= c0) & (cx < c0 + wc) & (cy >= c0) & (cy < c0 + wc)
    halo = (cx >= c0 - 1) & (cx <= c0 + wc) & (cy >= c0 - 1) & (cy <= c0 + wc)
    ids = np.nonzero(halo)[0]
    xl = (cx[ids] - c0 + 2).astype(np.float64) * h + ox[ids]
    yl = (cy[ids] - c0 + 2).astype(np.float64) * h + oy[ids]
    box = (wc + 6) * h + 10.0                        # no pair reaches across the wrap
    sub = np.nonzero(win[ids])[0]
    assert len(sub) > 15_000
    ofx, ofy, _, ofa = orc.forces_cells(xl, yl, box, subset=sub)
    fx, fy, _ = s.forces()
    gx, gy = fx[ids[sub]], fy[ids[sub]]
    oxs, oys, fas = ofx[sub], ofy[sub], ofa[sub]
    iso = fas == 0.0
    assert np.all(gx[iso] == 0.0) and np.all(gy[iso] == 0.0)
    # rounding allowance of the oracle's inputs (see the module docstring)
    from scipy.spatial import cKDTree

    pts = np.stack([xl, yl], axis=1)
    tree = cKDTree(pts)
    u = np.spacing(box) / 2.0
    delta = 2.0 * np.sqrt(2.0) * u + (2.0 * np.sqrt(2.0) * 2.0 ** -24 * 2.0 * h if fp32 else 0.0)
    allow = np.zeros(len(sub))
    for k, nb in enumerate(tree.query_ball_point(pts[sub], r=2.5)):
        d = pts[nb] - pts[sub[k]]
        r = np.hypot(d[:, 0], d[:, 1])
        r = r[(r > 0) & (r < 2.5)]
        f = 24.0 * (2.0 * r ** -13 - r ** -7)                 # F(r), sigma = eps = 1
        fp = 24.0 * (-26.0 * r ** -14 + 7.0 * r ** -8)        # F'(r)
        allow[k] = np.sum(np.abs(fp) + np.abs(f) / r) * delta
    scale = fas[~iso]
    ex = np.abs(gx[~iso] - oxs[~iso]) / (tol * scale + allow[~iso])
    ey = np.abs(gy[~iso] - oys[~iso]) / (tol * scale + allow[~iso])
    assert (~iso).sum() > len(sub) // 10             # enough interacting particles
    return float(max(ex.max(), ey.max()))        # <= 1 passes


def test_c3_fp64_vs_fp32_cell_offset(mdlg, orc):
    L = inputs.box_length(N, PHI)
    st = inputs.lattice_gas_state(N, L, T, seed=4_194_304)
    lx = int(round(L))
    res = {}
    for prec, tol, dbar in ((mdlg.MD_FP64, 1e-12, 5e-5), (mdlg.MD_FP32_CELLOFF, 1e-5, 1e-3)):
        p = mdlg.make_params(N, L, dt=5e-4, precision=prec, W=4, lg_every=(EVERY,), lx=(lx,))
        s = mdlg.System(p, st.x, st.y, st.vx, st.vy)
        e0 = s.energy()
        s.step(STEPS)
        s.sync()
        e1 = s.energy()
        drift = abs((e1[0] + e1[1]) - (e0[0] + e0[1])) / abs(e0[0] + e0[1])
        assert drift < dbar, (prec, drift)
        ferr = _forces_vs_oracle(s, orc, tol, prec == mdlg.MD_FP32_CELLOFF)
        assert ferr <= 1.0, (prec, ferr)
        P, _, stats = s.feq_measured(0, 0, 0)
        hist, ovf, nwin = s.hist_raw(0, 0, 0)
        assert nwin == STEPS // EVERY
        assert int(hist.sum()) + ovf == N * nwin
        res[prec] = (P, nwin, drift, ferr)
        s.close()
    P64, nwin, _, _ = res[mdlg.MD_FP64]
    P32 = res[mdlg.MD_FP32_CELLOFF][0]
    sigma = np.sqrt(np.maximum(P64 * (1.0 - P64), 1e-12) / (N * nwin))
    assert np.all(np.abs(P64 - P32) <= 6.0 * np.sqrt(2.0) * sigma + 1e-12), \
        np.max(np.abs(P64 - P32) / sigma)
