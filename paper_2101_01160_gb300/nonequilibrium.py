"""Non-equilibrium MDLG on local fields (Sec. 2; the outlook of Sec. 6): a
decaying shear wave in a batched ensemble of replicas, analysed through the
per-site occupation numbers n_i(x, t) of Eq. n_i, their ensemble average
f_i = <n_i> and the collision operator of Eq. mdlg_evolution.

Each replica is the dilute LJ gas (default phi = 0.0784, T = 20) started
with a transverse flow u_x(y) = U sin(2 pi y / L).  Every window of Delta t
the ensemble-summed occupation field is taken from the replicas' snapshots in
one call; from it, per lattice row y (the flow depends on y only), the
lattice velocity u(y) = sum_i v_i f_i / sum_i f_i and the covariance of the
lattice displacement components (the momentum flux), both fitted with
sin(k y), cos(k y) and a constant.

Python here sequences library calls and reduces the fields over rows:
MD, the fields, Xi, the global histogram and the shifted Gaussian run in
libmdlg.
"""

from __future__ import annotations

import json
import math

import numpy as np

from . import inputs, mdlg


def _fit_sine(prof, k, yc):
    A = np.stack([np.sin(k * yc), np.cos(k * yc), np.ones_like(yc)], axis=1)
    coef, *_ = np.linalg.lstsq(A, prof, rcond=None)
    return coef


def shear_wave(reps: int = 32, n: int = 16384, phi: float = 0.0784, T: float = 20.0,
               U: float = 2.0, dx_target: float = 10.0, dt: float = 5e-4, every: int = 2252,
               windows: int = 40, W: int = 4, seed: int = 500, eq_windows=(0, 10, 20, 39)) -> dict:
    """Runs the ensemble for `windows` windows of `every` MD steps and returns
    per-window results (lattice units: displacements per window in sites):
      amp[w]      fit of u(y): (sin, cos, constant) coefficients
      flux_cos[w] cos coefficient of cov(v_x, v_y)(y)
      a2[w]       thermal a^2: continuous second moment per axis / dx^2 less
                  the flow's share (mean over rows of u^2 / 2)
      xi_mass[w]  max over sites of |sum_i Xi_i| between windows w-1 and w
      hist_diff[w] entries where the field summed over sites differs from
                  mdlg_bin's global histogram of the same snapshots
      overflow[w] displacements outside the window
      uy_rms[w]   root mean square over rows of the lattice velocity u_y(y)
      gain[w]     for w in eq_windows, at rows with |sin| > 0.95: the
                  max-abs error of the unshifted Gaussian over that of the
                  Gaussian shifted by the row's lattice velocity
    plus the lattice (lx, dx), u_lat = U Delta t / dx and nu, the kinematic
    viscosity from the exponential decay of the sine amplitude."""
    import torch

    L = inputs.box_length(n, phi)
    lx = int(round(L / dx_target))
    sts = [inputs.shear_wave_state(n, L, T, U, seed=seed + r) for r in range(reps)]
    cat = [np.concatenate([getattr(s, f) for s in sts]) for f in ("x", "y", "vx", "vy")]
    p = mdlg.make_params(n, L, dt=dt, precision=mdlg.MD_FP32_CELLOFF, W=W, lg_every=(every,),
                         lx=(lx,))
    s = mdlg.System([p] * reps, *cat)
    ri = s.rep_info(0)
    ncell, h, dx = ri.ncell, ri.h, ri.dx_eff[0]
    side = 2 * W + 1
    vx = np.tile(np.arange(side) - W, side).astype(np.float64)      # class i -> (vx, vy)
    vy = np.repeat(np.arange(side) - W, side).astype(np.float64)
    k = 2.0 * math.pi / lx
    yc = np.arange(lx) + 0.5
    out = dict(amp=[], flux_cos=[], a2=[], xi_mass=[], hist_diff=[], overflow=[], uy_rms=[], gain={})
    prev = s.get_raw()
    last = None
    for w in range(windows):
        s.step(every)
        cur = s.get_raw()
        f, o = mdlg.site_occupation(*prev, *cur, ncell, h, lx, W)
        hist, ov, mom = mdlg.mdlg_bin(*prev, *cur, ncell, h, lx, W)
        out["hist_diff"].append(int((f.sum(dim=(1, 2)) != hist).sum().item()))
        out["overflow"].append(int(o.sum().item()) + int(ov.item()))
        out["xi_mass"].append(0 if last is None else
                              int(mdlg.collision(last, f, W).sum(dim=0).abs().max().item()))
        last = f
        F = f.cpu().numpy().astype(np.float64).sum(axis=2)          # [class, row]
        rho = F.sum(axis=0)
        ux = (vx[:, None] * F).sum(axis=0) / rho
        uy = (vy[:, None] * F).sum(axis=0) / rho
        pxy = (vx[:, None] * vy[:, None] * F).sum(axis=0) / rho
        out["amp"].append(_fit_sine(ux, k, yc).tolist())
        out["flux_cos"].append(float(_fit_sine(pxy - ux * uy, k, yc)[1]))
        a2 = float(mom[0].item()) / (2.0 * reps * n * dx * dx) - float(np.mean(ux ** 2)) / 2.0
        out["a2"].append(a2)
        out["uy_rms"].append(float(np.sqrt(np.mean(uy ** 2))))
        if w in eq_windows:
            g0 = mdlg.feq_gaussian(a2, 0.0, 0.0, W).cpu().numpy()
            gains = []
            for r in np.where(np.abs(np.sin(k * yc)) > 0.95)[0]:
                P = F[:, r] / rho[r]
                gu = mdlg.feq_gaussian(a2, float(ux[r]), 0.0, W).cpu().numpy()
                gains.append(float(np.max(np.abs(P - g0)) / np.max(np.abs(P - gu))))
            out["gain"][w] = gains
        prev = cur
    s.close()
    torch.cuda.synchronize()
    amp = np.array(out["amp"])[:, 0]
    t = (np.arange(windows) + 0.5) * every * dt
    slope = np.polyfit(t, np.log(np.maximum(amp, 1e-12)), 1)[0] if np.all(amp > 0) else float("nan")
    kp = 2.0 * math.pi / (lx * dx)
    out.update(lx=lx, dx=dx, u_lat=U * every * dt / dx, nu=float(-slope / kp ** 2),
               window_time=every * dt)
    return out


def main():
    import argparse

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--reps", type=int, default=32)
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--windows", type=int, default=40)
    ap.add_argument("--U", type=float, default=2.0)
    a = ap.parse_args()
    print(json.dumps(shear_wave(reps=a.reps, n=a.n, windows=a.windows, U=a.U)))


if __name__ == "__main__":
    main()
