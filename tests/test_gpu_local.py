"""GPU parity of the local MDLG fields (Sec. 2, Eqs. n_i and
mdlg_evolution) with the FP64 oracle, through the C ABI, and the
non-equilibrium check they exist for (paper_2101_01160_gb300.nonequilibrium).

Tolerances: occupation numbers, overflow and Xi bit-exact (lattice sites are
decided by the same operation-by-operation FP64 arithmetic on both sides);
Omega = scale * Xi exact (one product of an integer and a double).

The non-equilibrium case is a decaying shear wave, u_x(y) = U sin(2 pi y/L)
at t = 0, in a batched ensemble of replicas of the dilute LJ gas (phi =
0.0784, T = 20) sampled on a Table 1 lattice (Delta t = 1.1261, Delta x ~ 10):
the ensemble-summed fields give f_i = <n_i> and Omega_i = <Xi_i> per site.
Checks: every window's field sums to the global histogram of mdlg_bin on the
same snapshots; Xi conserves mass at every site; the row-averaged lattice
velocity is the imposed sine at U Delta t / Delta x, decaying; the
off-diagonal displacement moment (momentum flux) is in phase with -cos, the
sign of the shear rate; and the local distribution follows the Gaussian
shifted by the local velocity far better than the unshifted one.
"""

import math

import numpy as np
import pytest

from paper_2101_01160_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KEYS = ("cell0", "ox0", "oy0", "cell1", "ox1", "oy1")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pair(a, b):
    return dict(cell0=a["cell"], ox0=a["ox"], oy0=a["oy"], cell1=b["cell"], ox1=b["ox"], oy1=b["oy"])


@pytest.mark.parametrize("f64", [False, True])
@pytest.mark.parametrize("n", [0, 1, 1000, 262_147])
@pytest.mark.parametrize("lx,W", [(101, 4), (37, 1), (64, 10), (3, 4), (1, 0)])
def test_site_occupation_bitexact(mdlg, orc, f64, n, lx, W):
    ncell, h = 33, 101.283 / 33
    if not f64:
        h = float(np.float32(h))
    L = ncell * h
    s = inputs.random_celloff_snapshots(n, ncell, h, seed=n + lx + W, max_step=6.0, f64=f64,
                                        ties=min(n, 300), lattice_dx=L / lx)
    d = [_dev(s[k]) for k in KEYS]
    field, ovf = mdlg.site_occupation(*d, ncell, h, lx, W)
    torch.cuda.synchronize()
    rf, ro = orc.site_occupation(s, ncell, h, L, lx, W)
    assert np.array_equal(field.cpu().numpy(), rf)
    assert np.array_equal(ovf.cpu().numpy(), ro)
    # the field summed over its sites is mdlg_bin's histogram, bit for bit
    hist, ov, _ = mdlg.mdlg_bin(*d, ncell, h, lx, W)
    assert np.array_equal(field.sum(dim=(1, 2)).cpu().numpy(), hist.cpu().numpy())
    assert int(ovf.sum().item()) == int(ov.item())
    # accumulation: a second call adds the same counts
    mdlg.site_occupation(*d, ncell, h, lx, W, field=field, ovf=ovf)
    assert np.array_equal(field.cpu().numpy(), 2 * rf)
    assert np.array_equal(ovf.cpu().numpy(), 2 * ro)


@pytest.mark.parametrize("f64", [False, True])
def test_collision_bitexact_and_mass_conserving(mdlg, orc, f64):
    ncell, h, lx, W = 48, 2.75, 61, 3
    if not f64:
        h = float(np.float32(h))
    L = ncell * h
    walk = inputs.random_celloff_walk(300_001, ncell, h, seed=21, max_step=4.0, steps=2, f64=f64)
    fields = []
    for a, b in ((0, 1), (1, 2)):
        s = _pair(walk[a], walk[b])
        f, o = mdlg.site_occupation(*[_dev(s[k]) for k in KEYS], ncell, h, lx, W)
        rf, ro = orc.site_occupation(s, ncell, h, L, lx, W)
        assert np.array_equal(f.cpu().numpy(), rf) and int(o.sum().item()) == 0 == ro.sum()
        fields.append((f, rf))
    xi = mdlg.collision(fields[0][0], fields[1][0], W)
    om = mdlg.collision(fields[0][0], fields[1][0], W, scale=1.0 / 3.0)
    rxi = orc.collision(fields[0][1], fields[1][1], W)
    assert np.array_equal(xi.cpu().numpy(), rxi)
    assert np.array_equal(om.cpu().numpy(), rxi.astype(np.float64) * (1.0 / 3.0))
    assert not xi.sum(dim=0).any()
    assert int(xi.abs().sum().item()) > 0


def test_full_ensemble_size_bitexact(mdlg, orc):
    # the benchmark's configuration: 64 replicas of the standard system's
    # box (L = 1000) on Table 1's lx = 250 lattice, one call over all replicas
    n, ncell = 64 * 99_856, 333
    h = float(np.float32(1000.0 / ncell))
    L = ncell * h
    s = inputs.random_celloff_snapshots(n, ncell, h, seed=77, max_step=4.0, f64=False,
                                        ties=10_000, lattice_dx=L / 250)
    field, ovf = mdlg.site_occupation(*[_dev(s[k]) for k in KEYS], ncell, h, 250, 4)
    rf, ro = orc.site_occupation(s, ncell, h, L, 250, 4)
    assert np.array_equal(field.cpu().numpy(), rf)
    assert np.array_equal(ovf.cpu().numpy(), ro)


def _near_lines(rng, m, ncell, h, lx):
    """Positions on lattice lines j dx and 1-3 ulps to either side, encoded
    as (cell, FP64 offset)."""
    L = ncell * h
    dxl = L / lx
    j = rng.integers(0, lx, m)
    x = j * dxl
    for k in range(m):
        for _ in range(int(rng.integers(0, 4))):
            x[k] = np.nextafter(x[k], np.inf if k % 2 else -np.inf)
    x = np.where(x < 0, x + L, x)
    c = np.clip(np.floor(x / h).astype(np.int64), 0, ncell - 1)
    return c, x - c * h


@pytest.mark.parametrize("lx", [101, 250, 37, 7])
def test_lattice_line_neighbours_bitexact(mdlg, orc, lx):
    # the product x * (1/dx) decides the cell only away from lattice lines;
    # on and next to them the division decides, exactly as in the oracle
    ncell, h, W, m = 333, 1000.0 / 333, 4, 200_000
    rng = np.random.Generator(np.random.PCG64(lx))
    cx0, ox0 = _near_lines(rng, m, ncell, h, lx)
    cy0, oy0 = _near_lines(rng, m, ncell, h, lx)
    cx1, ox1 = _near_lines(rng, m, ncell, h, lx)
    cy1, oy1 = _near_lines(rng, m, ncell, h, lx)
    s = dict(cell0=(cy0 * ncell + cx0).astype(np.int32), ox0=ox0, oy0=oy0,
             cell1=(cy1 * ncell + cx1).astype(np.int32), ox1=ox1, oy1=oy1)
    d = [_dev(s[k]) for k in KEYS]
    field, ovf = mdlg.site_occupation(*d, ncell, h, lx, W)
    rf, ro = orc.site_occupation(s, ncell, h, ncell * h, lx, W)
    assert np.array_equal(field.cpu().numpy(), rf)
    assert np.array_equal(ovf.cpu().numpy(), ro)
    hist, ov, _ = mdlg.mdlg_bin(*d, ncell, h, lx, W)
    rh, rov, _ = orc.bin_celloff(s, ncell, h, ncell * h, lx, W)
    assert np.array_equal(hist.cpu().numpy().astype(np.int64), rh) and int(ov.item()) == rov


def test_rejects_bad_arguments(mdlg):
    import ctypes as C

    z = torch.zeros(8, dtype=torch.int32, device="cuda")
    f = torch.zeros(8, dtype=torch.float32, device="cuda")
    # the binding refuses before any call ...
    for lx, W in ((0, 1), (4, 11), (20_000, 10)):                   # lx < 1, W > MD_MAX_W, too large
        with pytest.raises(ValueError):
            mdlg.site_occupation(z, f, f, z, f, f, 2, 1.0, lx, W)
    with pytest.raises(ValueError):                                  # field of the wrong shape
        mdlg.site_occupation(z, f, f, z, f, f, 2, 1.0, 4, 1, field=z)
    n = torch.zeros((9, 3, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        mdlg.collision(n, n, 11)
    with pytest.raises(ValueError):                                  # W does not match the class count
        mdlg.collision(n, n, 2)
    # ... and so does the C ABI itself, before a launch (the outputs are never touched)
    lib = mdlg.load()
    s0 = mdlg.md_snapshot(z.data_ptr(), f.data_ptr(), f.data_ptr(), 0, 2, 1.0)
    for lx, W, code in ((0, 1, mdlg.MD_E_ARG), (4, 11, mdlg.MD_E_ARG), (20_000, 10, mdlg.MD_E_LIMIT)):
        rc = lib.mdlg_site_occupation(C.byref(s0), C.byref(s0), 8, lx, W, mdlg._ptr(z), mdlg._ptr(z), None)
        assert rc == code, (lx, W, rc)
    assert lib.mdlg_collision(mdlg._ptr(n), mdlg._ptr(n), 3, 11, 1.0, mdlg._ptr(n), None, None) == mdlg.MD_E_ARG
    assert lib.mdlg_collision(mdlg._ptr(n), mdlg._ptr(n), 3, 1, 1.0, None, None, None) == mdlg.MD_E_ARG
    torch.cuda.synchronize()


def test_shear_wave_ensemble(mdlg):
    from paper_2101_01160_gb300 import nonequilibrium

    nwin = 40
    r = nonequilibrium.shear_wave(reps=32, n=16384, U=2.0, windows=nwin, eq_windows=(10, 20, 39))
    # exact identities on every window
    assert max(r["hist_diff"]) == 0 and max(r["overflow"]) == 0
    assert max(r["xi_mass"]) == 0
    amp = np.array(r["amp"])
    u_lat = r["u_lat"]
    # the imposed sine, at the imposed amplitude, no cosine part, no mean
    assert abs(amp[0, 0] / u_lat - 1.0) < 0.1, (amp[0, 0], u_lat)
    assert np.all(np.abs(amp[:, 1]) < 0.05 * u_lat) and np.all(np.abs(amp[:, 2]) < 0.02 * u_lat)
    # decay: every window positive, the last quarter below the first
    q = nwin // 4
    assert np.all(amp[:, 0] > 0)
    assert amp[-q:, 0].mean() < 0.97 * amp[:q, 0].mean(), amp[:, 0]
    assert r["nu"] > 0
    # momentum flux in phase with -cos (the shear rate goes as +cos)
    fc = np.array(r["flux_cos"])
    assert fc.mean() < 0 and abs(fc.mean()) > 5 * fc.std() / math.sqrt(nwin), fc
    # once the lattice start has mixed (no mean u_y), the Gaussian shifted by
    # the local velocity fits the local distribution much better
    # (per-row sampling noise of u_y is about 0.02 u_lat at this ensemble size)
    assert max(r["uy_rms"][10:]) < 0.05 * u_lat
    assert min(min(g) for g in r["gain"].values()) > 3.0, r["gain"]
