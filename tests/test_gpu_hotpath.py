"""GPU parity of the headline path itself against the FP64 oracle, through
the C-ABI: the Verlet-list forces that every MD step sums (Sec. 4), the fused
sampling of an uneven multi-replica batch in the bench's launch shape
(Sec. 2, Eq. n_i, and the moments of Sec. 3(b)), the energy and momentum
readout, and the normalisation and symmetric-set averaging of the measured
equilibrium (Eq. theory_feq, Sec. 5).

Bars (the allowances are derived in _bars.py):
  * forces: |F - F_oracle| <= tol * sum_j |F_ij| + rounding allowance,
    tol = 1e-12 (FP64), 1e-5 (FP32 cell + offset);
  * histograms and overflow: bit-exact;
  * moment sums: the displacement forms of the two sides differ by at most
    2 ulp(L), propagated to the sums, plus FP64 summation bounds;
  * kinetic energy and momentum: 1e-12 relative (the same velocities summed
    in another order); potential energy: 1e-12 of sum|pe_i| (FP64), 1e-5 of
    it plus the pair allowance (FP32);
  * P = H / (N windows): bit-exact (one IEEE division on both sides); its
    symmetric-set average: 4 2^-53 relative (sum and divide in another
    order).
"""

import numpy as np
import pytest

from paper_2101_01160_gb300 import inputs
import _bars as fc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS = fc.EPS


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_list_forces_match_oracle_through_a_rebuild_cycle(mdlg, orc, prec, tol):
    """Forces of the step kernel's own force pass (Verlet lists, built up to
    one rebuild interval earlier, the skin nearly used up just before each
    rebuild) at every step of more than one rebuild cycle."""
    n, phi, T = 30_000, 0.25, 5.0
    L = inputs.box_length(n, phi)
    st = inputs.lattice_gas_state(n, L, T, seed=31)
    p = mdlg.make_params(n, L, precision=prec, lg_every=(100,), lx=(int(round(L)),), skin=0.4)
    s = mdlg.System(p, st.x, st.y, st.vx, st.vy)
    s.step(200)
    info = s.rep_info(0)
    nc, h, Le = int(info.ncell), float(info.h), float(info.L_eff)
    r0 = s.info().n_rebuilds
    worst = 0.0
    for _ in range(70):
        cell, ox, oy = (t.cpu().numpy() for t in s.get_raw())
        gx, gy = s.step_forces(1)
        x, y = fc.decode(cell, ox, oy, nc, h)
        ofx, ofy, _, ofa = orc.forces_cells(x, y, Le)
        allow = fc.force_allowance(x, y, Le, h, prec == mdlg.MD_FP32_CELLOFF)
        worst = max(worst, fc.force_ratio(gx, gy, ofx, ofy, ofa, allow, tol))
        assert (ofa > 0).sum() > n // 2
    assert worst <= 1.0, worst
    assert s.info().n_rebuilds - r0 >= 1          # the steps span a rebuild
    s.close()


def _uneven_batch(mdlg, R=16, seed=11, prec=1):
    Ns, phis, Ts = inputs.ensemble_params(R, seed=seed)
    params, cat = [], [[], [], [], []]
    for r in range(R):
        L = inputs.box_length(int(Ns[r]), float(phis[r]))
        st = inputs.lattice_gas_state(int(Ns[r]), L, float(Ts[r]), seed=900 + r)
        params.append(mdlg.make_params(int(Ns[r]), L, precision=prec, W=4, lg_every=(100, 250),
                                       lx=(int(round(L)), int(round(L / 2))), skin=0.4))
        for a, f in zip(cat, ("x", "y", "vx", "vy")):
            a.append(getattr(st, f))
    return params, [np.concatenate(a) for a in cat]


def test_fused_sampling_uneven_batch_bench_shape(mdlg, orc):
    """16 replicas of uneven N, phi and T (the bench's draw recipe, about
    360k particles) in the bench's launch shape (256 threads, one chunk per
    thread, global staging, full-occupancy registers, full resident grid, so
    that CTAs own chunks of several replicas): per replica, interval and
    lattice, the histogram and overflow increments of one window equal the
    oracle's binning of the kernel's own snapshots, and the moment sums
    agree within their bar."""
    params, cat = _uneven_batch(mdlg)
    s = mdlg.System(params, *cat)
    s.tune(256, 1, 3)
    R = len(params)
    ns = [p.n for p in params]
    base = np.concatenate([[0], np.cumsum(ns)])
    s.step(500)
    snaps = {k: [t.cpu().numpy() for t in s.get_snapshot(k)] for k in (0, 1)}
    before = {(r, k, d): s.hist_raw(r, k, d) for r in range(R) for k in (0, 1) for d in (0, 1)}
    mom0 = {(r, k): fc.moment_sums(s, r, k, ns[r]) for r in range(R) for k in (0, 1)}
    checked = 0
    for k, adv in ((0, 100), (1, 150)):      # one window of interval k ends at 600 / 750
        s.step(adv)
        after = [t.cpu().numpy() for t in s.get_snapshot(k)]
        for r in range(R):
            info = s.rep_info(r)
            nc, h, Le = int(info.ncell), float(info.h), float(info.L_eff)
            sl = slice(base[r], base[r + 1])
            b = [a[sl] for a in snaps[k]]
            a_ = [a[sl] for a in after]
            sn = dict(cell0=b[0], ox0=b[1], oy0=b[2], cell1=a_[0], ox1=a_[1], oy1=a_[2])
            for d in (0, 1):
                h1, o1, w1 = s.hist_raw(r, k, d)
                h0, o0, w0 = before[(r, k, d)]
                assert w1 == w0 + 1
                rh, ro, rm = orc.bin_celloff(sn, nc, h, Le, params[r].lx[d], 4)
                assert np.array_equal(h1 - h0, rh), (r, k, d)
                assert o1 - o0 == ro
                checked += 1
            S1 = fc.moment_sums(s, r, k, ns[r])
            (S2, S4), (b2, b4) = fc.moment_bar(b, a_, nc, h, Le, mom0[(r, k)], S1)
            inc = S1 - mom0[(r, k)]
            assert abs(inc[0] - S2) <= b2, (r, k, inc[0], S2, b2)
            assert abs(inc[1] - S4) <= b4, (r, k, inc[1], S4, b4)
            assert abs(rm[0] - S2) <= 1e-9 * S2        # the oracle's own sums agree
    assert checked == R * 2 * 2
    s.close()


def test_dynamic_tail_bit_identical_to_dealt_chunks(mdlg):
    """Global-memory launch shapes deal the first rounds of chunks to CTAs
    and let CTAs claim the rest each step; a claimed chunk's neighbour list
    was built by another CTA in the last rebuild.  Over many rebuilds of an
    uneven batch large enough to have a claimed tail (about 30k particles
    per replica, 48 replicas, so more than two rounds of chunks), the state,
    histograms and rebuild count equal those of the staged shape, which
    claims nothing."""
    params, cat = _uneven_batch(mdlg, R=48, seed=23)
    out = []
    for shape in ((256, 1, 1), (256, 1, 3), (128, 1, 2)):
        s = mdlg.System(params, *cat)
        s.tune(*shape)
        for _ in range(3):
            s.step(300)
        s.sync()
        out.append((s.get_state(), [s.hist_raw(r, 0, 0)[0] for r in range(0, len(params), 5)],
                    s.info().n_rebuilds))
        s.close()
    assert out[0][2] >= 20, out[0][2]
    for o in out[1:]:
        for u, v in zip(out[0][0], o[0]):
            assert np.array_equal(u, v)
        for u, v in zip(out[0][1], o[1]):
            assert np.array_equal(u, v)
        assert o[2] == out[0][2]


@pytest.mark.parametrize("prec", [0, 1])
def test_energy_matches_oracle(mdlg, orc, prec):
    """md_energy of each replica equals the oracle's kinetic energy, shifted
    potential energy and momentum on the same state; md_energy_batch gives
    every replica's four values bit for bit."""
    spec = [(3000, 0.25, 2.0), (5000, 0.08, 20.0), (4000, 0.15, 1.0)]
    params, cat = [], [[], [], [], []]
    for r, (n, phi, T) in enumerate(spec):
        L = inputs.box_length(n, phi)
        st = inputs.lattice_gas_state(n, L, T, seed=60 + r)
        params.append(mdlg.make_params(n, L, precision=prec, lg_every=(100,), lx=(int(L),)))
        for a, f in zip(cat, ("x", "y", "vx", "vy")):
            a.append(getattr(st, f))
    s = mdlg.System(params, *[np.concatenate(a) for a in cat])
    s.step(300)
    x, y, vx, vy = s.get_state()
    cell, ox, oy = (t.cpu().numpy() for t in s.get_raw())
    base = 0
    eb = s.energy_batch()
    assert eb.shape == (len(spec), 4)
    for r, (n, _, _) in enumerate(spec):
        info = s.rep_info(r)
        nc, h, Le = int(info.ncell), float(info.h), float(info.L_eff)
        sl = slice(base, base + n)
        base += n
        g = s.energy(r)
        assert np.array_equal(eb[r], g), (r, eb[r], g)
        o = orc.energy(x[sl], y[sl], vx[sl], vy[sl], Le)
        assert abs(g[0] - o[0]) <= 1e-12 * o[0]
        pabs = np.sum(np.abs(vx[sl])), np.sum(np.abs(vy[sl]))
        assert abs(g[2] - o[2]) <= 1e-12 * pabs[0] and abs(g[3] - o[3]) <= 1e-12 * pabs[1]
        # potential energy from the raw encoding, as the kernels hold it
        xr, yr = fc.decode(cell[sl], ox[sl], oy[sl], nc, h)
        _, _, pe, _ = orc.forces_cells(xr, yr, Le)
        fp32 = prec == mdlg.MD_FP32_CELLOFF
        bar = (1e-5 if fp32 else 1e-12) * np.sum(np.abs(pe)) + fc.energy_allowance(xr, yr, Le, h, fp32)
        assert abs(g[1] - pe.sum()) <= bar, (r, g[1], pe.sum(), bar)
        assert abs(o[1] - pe.sum()) <= bar
    s.close()


def test_normalisation_and_symmetrisation_match_oracle(mdlg, orc):
    """Device normalisation P = H / (N windows) and the symmetric-set
    averages of feq_measured and feq_batch against the integer histogram
    normalised here and the oracle's symmetrisation, element by element."""
    params, cat = _uneven_batch(mdlg, R=6, seed=12)
    s = mdlg.System(params, *cat)
    s.step(1000)
    for k in (0, 1):
        Pb, _, _, stats = mdlg.feq_batch(s, k, 1, symmetrize=True)
        for r, p in enumerate(params):
            H, ovf, nwin = s.hist_raw(r, k, 1)
            ref = H / (float(p.n) * float(nwin))
            P, _, st = s.feq_measured(r, k, 1)
            assert np.array_equal(P, ref), (r, k)
            assert st.n_windows == nwin and st.n_overflow == ovf
            assert int(H.sum()) + ovf == p.n * nwin
            sym = orc.symmetrize(ref, 4)
            Ps, _, _ = s.feq_measured(r, k, 1, symmetrize=True)
            assert np.all(np.abs(Ps - sym) <= 4 * EPS * sym), (r, k)
            assert np.all(np.abs(Pb[r] - sym) <= 4 * EPS * sym), (r, k)
            assert stats[r, 8] == nwin and stats[r, 10] == ovf
    s.close()
