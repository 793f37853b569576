"""Reproduction of the paper's simulation setup (Table 1, Sec. 4) and of the
comparison of Sec. 5 (Figs. 3-5): for each (Delta t, Delta x) row of Table
1, the measured equilibrium averaged over the D2Q25 symmetric sets, against
the single Gaussian and the Poisson WSG equilibria at the measured moments.

The system is the paper's standard one: N = 99,856 particles in a periodic
box of L = 1000 sigma (phi = 0.0784), T = 20, LJ truncated and shifted at
rc = 2.5, started from the seeded jittered-lattice state.  Per row the paper
takes 2000 sampling windows from one run at MD step 1e-4; here the MD step
is a parameter and the windows are split over `reps` independent replicas
run as one batched ensemble (same statistics, more parallel work).  Table
1's rows are grouped four at a time into one system each (four sampling
intervals x four lattices, of which the diagonal pairs are used).  Row 3 is
printed as 5.5 x 180; the run uses lx = 180 (Delta x = L/180 = 5.5(5)),
the reading that keeps lx Delta x = L and gives the table's a^2.

Python here only sequences library calls and pools the replicas' results:
MD, binning, the measured f_eq, lambda, the analytic equilibria and their
comparison run in libmdlg.
"""

from __future__ import annotations

import json
import time

import numpy as np

from . import inputs, mdlg

N, L, T = 99_856, 1000.0, 20.0
A2_TABLE = 0.1611            # Sec. 4: a^2 held fixed over the rows of Table 1
# Table 1: coarse-grained time step Delta t and lattice points lx (Delta x = L / lx)
TABLE1 = ((0.3911, 250), (0.5000, 200), (0.5626, 180), (0.6927, 150), (0.9009, 120),
          (1.1261, 100), (1.4994, 80), (1.6342, 75), (2.0338, 64), (2.9280, 50),
          (4.1821, 40), (6.1751, 32))
# D2Q25 symmetric sets by (|vx|, |vy|): f0, f1-4, f5-8, f9-12, f13-20, f21-24
SETS = ((0, 0), (0, 1), (1, 1), (0, 2), (1, 2), (2, 2))
SET_NAMES = ("f0", "f1-4", "f5-8", "f9-12", "f13-20", "f21-24")


def set_means(P, W=4):
    """Mean of P over each D2Q25 symmetric set (P indexed [vy][vx], v in -W..W)."""
    side = 2 * W + 1
    P = np.asarray(P).reshape(side, side)
    out = []
    for a, b in SETS:
        vals = [P[vy + W, vx + W] for vy in range(-W, W + 1) for vx in range(-W, W + 1)
                if sorted((abs(vx), abs(vy))) == [a, b]]
        out.append(float(np.mean(vals)))
    return np.array(out)


def _pool(sys_, n_rep, k):
    """Pools the replicas' results for interval k on lattice k: P and the
    raw moments weighted by each replica's sample count (exact pooling of
    the means)."""
    Ps, w, mu2, mu4 = [], [], [], []
    ov = 0
    nw = 0
    for r in range(n_rep):
        P, _, st = sys_.feq_measured(r, k, k, symmetrize=True)
        Ps.append(P)
        w.append(st.n_samples)
        mu2.append(st.mu2)
        mu4.append(st.mu4)
        ov += st.n_overflow
        nw += st.n_windows
        dx = st.dx_eff
    w = np.asarray(w, np.float64)
    P = (np.asarray(Ps) * w[:, None]).sum(0) / w.sum()
    return (P, float(np.dot(w, mu2) / w.sum()), float(np.dot(w, mu4) / w.sum()), dx,
            int(w.sum()), ov, nw)


def run(windows: int = 200, reps: int = 1, n_equil: int = 40_000, dt: float = 5e-4,
        seed: int = 1, rows=range(len(TABLE1))) -> list:
    """Runs the given Table 1 rows (0-based), four per batched system of
    `reps` replicas, each replica sampling `windows` windows of the longest
    interval of its group.  Returns one dict per row."""
    import torch

    rows = list(rows)
    out = []
    for g in range(0, len(rows), 4):
        grp = rows[g:g + 4]
        every = tuple(int(round(TABLE1[r][0] / dt)) for r in grp)
        lx = tuple(TABLE1[r][1] for r in grp)
        p = mdlg.make_params(N, L, dt=dt, precision=mdlg.MD_FP32_CELLOFF, W=4, n_equil=n_equil,
                             lg_every=every, lx=lx)
        sts = [inputs.lattice_gas_state(N, L, T, seed=1000 * seed + 37 * g + r)
               for r in range(reps)]
        cat = [np.concatenate([getattr(s, f) for s in sts]) for f in ("x", "y", "vx", "vy")]
        s = mdlg.System([p] * reps, *cat)
        s.autotune(100)
        nsteps = n_equil + windows * max(every)
        t0 = time.perf_counter()
        s.step(nsteps)
        s.sync()
        wall = time.perf_counter() - t0
        for k, r in enumerate(grp):
            P, mu2, mu4, dx, nsamp, ov, nw = _pool(s, reps, k)
            a2 = mu2 / dx ** 2
            lam_t, rc = mdlg.wsg_lambda(mu2, mu4, allow_domain=True)
            lam = float(lam_t.item()) if rc == 0 else 0.0
            Gd = mdlg.feq_gaussian(a2)
            Wd = mdlg.feq_wsg(a2, lam)
            Pd = torch.as_tensor(P, device="cuda")
            cg = mdlg.feq_compare(Pd, Gd).cpu().numpy()
            cw = mdlg.feq_compare(Pd, Wd).cpu().numpy()
            sm, sg, sw = set_means(P), set_means(Gd.cpu().numpy()), set_means(Wd.cpu().numpy())
            out.append({
                "row": r + 1, "dt_lg": TABLE1[r][0], "dx": dx, "lx": lx[k],
                "interval_steps": every[k], "windows": nw, "samples": nsamp,
                "a2": a2, "kurtosis": mu4 / mu2 ** 2, "lambda": lam, "lambda_status": rc,
                "md_over_g": (sm / sg).tolist(), "wsg_over_g": (sw / sg).tolist(),
                "max_abs_md_g": float(cg[0]), "kl_md_g": float(cg[1]),
                "max_abs_md_wsg": float(cw[0]), "kl_md_wsg": float(cw[1]),
                "overflow_frac": ov / max(1, nsamp),
                "group_particle_steps": float(N) * reps * nsteps, "group_wall_s": wall,
            })
        s.close()
    return out


def main():
    import argparse

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--windows", type=int, default=200, help="windows per replica")
    ap.add_argument("--reps", type=int, default=1, help="replicas per row group")
    ap.add_argument("--n-equil", type=int, default=40_000)
    ap.add_argument("--dt", type=float, default=5e-4, help="MD step (tau)")
    ap.add_argument("--seed", type=int, default=1)
    a = ap.parse_args()
    res = run(windows=a.windows, reps=a.reps, n_equil=a.n_equil, dt=a.dt, seed=a.seed)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
