"""Force, energy and moment bars of the GPU parity tests (imported by test
files).

The oracle evaluates the FP64 Lennard-Jones force (Sec. 4) from a GPU state
in the snapshot encoding: position = cell * h + offset in FP64, in the
periodic box of edge ncell * h with the minimum image.  The bar per particle
and axis is

    |F_gpu - F_oracle| <= tol * sum_j |F_ij| + allowance,

tol = 1e-12 (FP64) or 1e-5 (FP32).  The allowance is the effect of input
rounding on each pair force F(r) r_hat: (|F'(r)| + |F(r)| / r) * delta per
pair, delta = 2 sqrt(2) u for the oracle's own decoded coordinates (u = half
an ulp of the box edge), plus in FP32 2 sqrt(2) 2^-24 2h for the kernel's
pair vector dcell * h + (off_j - off_i), two roundings of magnitude <= 2h.
Near the zero of the LJ force (r ~ 1.12) these terms dominate sum_j |F_ij|.
"""

import numpy as np


def decode(cell, ox, oy, ncell, h):
    cell = np.asarray(cell).astype(np.int64)
    cx, cy = cell % ncell, cell // ncell
    x = cx.astype(np.float64) * h + np.asarray(ox).astype(np.float64)
    y = cy.astype(np.float64) * h + np.asarray(oy).astype(np.float64)
    return x, y


def _pairs(x, y, box, rc):
    from scipy.spatial import cKDTree

    pts = np.stack([np.mod(x, box), np.mod(y, box)], axis=1)
    pts[pts >= box] -= box
    tree = cKDTree(pts, boxsize=box)
    ij = tree.query_pairs(r=rc, output_type="ndarray")
    d = pts[ij[:, 1]] - pts[ij[:, 0]]
    d -= box * np.round(d / box)
    r = np.hypot(d[:, 0], d[:, 1])
    keep = (r > 0) & (r < rc)
    return ij[keep], r[keep]


def delta(box, h, fp32):
    u = np.spacing(box) / 2.0
    return 2.0 * np.sqrt(2.0) * u + (2.0 * np.sqrt(2.0) * 2.0 ** -24 * 2.0 * h if fp32 else 0.0)


def force_allowance(x, y, box, h, fp32, rc=2.5):
    """Per-particle rounding allowance of the force bar (module docstring)."""
    ij, r = _pairs(x, y, box, rc)
    f = 24.0 * (2.0 * r ** -13 - r ** -7)              # F(r), sigma = eps = 1
    fp = 24.0 * (-26.0 * r ** -14 + 7.0 * r ** -8)     # F'(r)
    a = (np.abs(fp) + np.abs(f) / r) * delta(box, h, fp32)
    out = np.zeros(len(x))
    np.add.at(out, ij[:, 0], a)
    np.add.at(out, ij[:, 1], a)
    return out


def energy_allowance(x, y, box, h, fp32, rc=2.5):
    """Bound on the rounding of the summed pair energy: |V'(r)| delta per
    pair (V = 4 (r^-12 - r^-6)), plus in FP32 the relative rounding of each
    pair's terms, 32 2^-24 (s^6 carries at most 16 2^-24 with the
    approximate reciprocal, s^12 twice that) times 4 (r^-12 + r^-6) + |V(rc)|."""
    ij, r = _pairs(x, y, box, rc)
    vp = 24.0 * (-2.0 * r ** -13 + r ** -7)
    vc = 4.0 * (rc ** -12 - rc ** -6)
    a = np.abs(vp) * delta(box, h, fp32)
    if fp32:
        a = a + 32.0 * 2.0 ** -24 * (4.0 * (r ** -12 + r ** -6) + abs(vc))
    return float(a.sum())


def force_ratio(gx, gy, ox, oy, ofa, allow, tol):
    """max over particles and axes of |F_gpu - F_oracle| / bar (<= 1 passes);
    an isolated particle's force must be exactly 0."""
    iso = ofa == 0.0
    assert np.all(gx[iso] == 0.0) and np.all(gy[iso] == 0.0)
    bar = tol * ofa[~iso] + allow[~iso]
    ex = np.abs(gx[~iso] - ox[~iso]) / bar
    ey = np.abs(gy[~iso] - oy[~iso]) / bar
    return float(max(ex.max(initial=0.0), ey.max(initial=0.0)))


EPS = 2.0 ** -53


def moment_bar(s0, s1, nc, h, L, S_before, S_after):
    """Oracle values and bars of the increments of the two displacement-moment
    sums over one window (Sec. 3(b)), from the snapshots (cell, off_x, off_y)
    s0 and s1.  The kernel forms the displacement in the cell frame, the
    oracle from decoded positions: the two differ by at most 2 ulp(L)
    (delta), so |dS2| <= 2 delta sum|d| and |dS4| <= 4 delta sum|d|^3; plus
    the FP64 summation bound m 2^-53 S of either order over m terms, and
    8 2^-53 (|S_before| + |S_after|) for reading the running sums back
    through mu_k = S / (2 N windows).  Returns ((S2, S4), (bar2, bar4))."""
    x0, y0 = decode(s0[0], s0[1], s0[2], nc, h)
    x1, y1 = decode(s1[0], s1[1], s1[2], nc, h)
    d = np.concatenate([x1 - x0, y1 - y0])
    d -= L * np.round(d / L)
    a = np.abs(d)
    dl = 2.0 * np.spacing(L)
    S2, S4 = float(np.sum(d ** 2)), float(np.sum(d ** 4))
    m = len(d)
    b2 = 2 * dl * a.sum() + m * EPS * S2 + 8 * EPS * (abs(S_before[0]) + abs(S_after[0]))
    b4 = 4 * dl * np.sum(a ** 3) + m * EPS * S4 + 8 * EPS * (abs(S_before[1]) + abs(S_after[1]))
    return (S2, S4), (b2, b4)


def moment_sums(system, r, k, n):
    """Running sums (S2, S4) of replica r, interval k, read back from
    feq_measured's mu2 and mu4."""
    _, _, st = system.feq_measured(r, k, 0)
    return np.array([st.mu2, st.mu4]) * 2.0 * n * st.n_windows
