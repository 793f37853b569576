"""GPU parity of the displacement-PDF diagnostics (Sec. 3(b), Fig. 2) with
the FP64 oracle, through the C ABI.

Tolerances: histogram counts bit-exact (the displacement and the bin index
are rounded operation by operation on both sides); Gaussian and WSG bin
masses 1e-12 absolute (same closed forms, erf and Poisson weights evaluated
in a different order); K(X_i) 1e-14 relative.
"""

import math

import numpy as np
import pytest

from paper_2101_01160_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


KEYS = ("cell0", "ox0", "oy0", "cell1", "ox1", "oy1")


@pytest.mark.parametrize("f64", [False, True])
@pytest.mark.parametrize("n", [0, 1, 1000, 262_147])
def test_disp_hist_bitexact(mdlg, orc, f64, n):
    ncell, h = 33, 101.283 / 33
    if not f64:
        h = float(np.float32(h))
    s = inputs.random_celloff_snapshots(n, ncell, h, seed=n + 11, max_step=6.0, f64=f64,
                                        ties=min(n, 300), lattice_dx=ncell * h / 101)
    for width, nbins in ((0.05, 64), (0.25, 200), (1.0 / 64, 8192), (2.0, 3)):
        hist, out = mdlg.disp_hist(*[_dev(s[k]) for k in KEYS], ncell, h, width, nbins)
        torch.cuda.synchronize()
        rh, ro = orc.disp_hist(s, ncell, h, ncell * h, width, nbins)
        assert np.array_equal(hist.cpu().numpy(), rh)
        assert int(out.item()) == ro
        assert int(hist.sum().item()) + ro == 2 * n


def test_disp_hist_edges_and_wrap(mdlg, orc):
    # exact binary values: displacements on bin edges go to the upper bin;
    # one pair crosses the periodic boundary; one displacement is outside
    ncell, h = 8, 2.0
    pos = [(1.0, 1.0, 1.25, 0.75), (15.75, 3.0, 0.25, 3.75), (4.0, 4.0, 7.0, 4.0)]
    s = {k: [] for k in KEYS}
    for x0, y0, x1, y1 in pos:
        for t, (x, y) in (("0", (x0, y0)), ("1", (x1, y1))):
            cx, cy = int(x // h), int(y // h)
            s["cell" + t].append(cy * ncell + cx)
            s["ox" + t].append(x - cx * h)
            s["oy" + t].append(y - cy * h)
    s = {k: np.array(v, dtype=np.int32 if k.startswith("cell") else np.float64) for k, v in s.items()}
    hist, out = mdlg.disp_hist(*[_dev(s[k]) for k in KEYS], ncell, h, 0.25, 8)
    rh, ro = orc.disp_hist(s, ncell, h, ncell * h, 0.25, 8)
    assert np.array_equal(hist.cpu().numpy(), rh) and int(out.item()) == ro == 1


@pytest.mark.parametrize("f64", [False, True])
def test_disp_hist_bin_edges_ulps(mdlg, orc, f64):
    """Displacements placed on bin edges k * width and 1-3 ulp of the stored
    offset to either side: the GPU bin of floor(delta / width) equals the
    oracle's on every one (the FP32 decision's guard sends these to the FP64
    division)."""
    ft = np.float64 if f64 else np.float32
    ncell, nbins = 64, 512
    h = float(ft(3.1))
    rng = np.random.default_rng(21 + f64)
    n = 7 * 4096
    for width in (0.05, 0.25, 1.0 / 3.0):
        c0 = rng.integers(0, ncell * ncell, n)
        o0x = rng.uniform(0.0, h, n).astype(ft)
        o0y = rng.uniform(0.0, h, n).astype(ft)
        k = rng.integers(-nbins // 2 + 1, nbins // 2 - 1, (2, n))
        dc = rng.integers(-2, 3, (2, n))
        m = np.repeat(np.arange(-3, 4), n // 7)            # ulps from the edge
        o1 = []
        for ax, o0 in enumerate((o0x, o0y)):
            target = k[ax] * width - dc[ax] * h + o0.astype(np.float64)
            v = target.astype(ft)
            for step in range(3):                         # walk m ulps away
                up = m > step
                dn = m < -step
                v = np.where(up, np.nextafter(v, ft(np.inf)), v)
                v = np.where(dn, np.nextafter(v, ft(-np.inf)), v)
            o1.append(v.astype(ft))
        cx0, cy0 = c0 % ncell, c0 // ncell
        cx1 = (cx0 + dc[0]) % ncell
        cy1 = (cy0 + dc[1]) % ncell
        sn = dict(cell0=c0.astype(np.int32), ox0=o0x, oy0=o0y,
                  cell1=(cy1 * ncell + cx1).astype(np.int32), ox1=o1[0], oy1=o1[1])
        hist, outc = mdlg.disp_hist(*[_dev(sn[kk]) for kk in KEYS], ncell, h, width, nbins)
        rh, ro = orc.disp_hist(sn, ncell, h, ncell * h, width, nbins)
        assert np.array_equal(hist.cpu().numpy(), rh), width
        assert int(outc.item()) == ro
        # the edges really are hit: the displacements straddle them
        d = dc[0] * h + (o1[0].astype(np.float64) - o0x.astype(np.float64))
        assert np.mean(np.floor(d / width) == k[0]) > 0.3
        assert np.mean(np.floor(d / width) == k[0] - 1) > 0.3


def test_disp_hist_rejects_bad_args(mdlg):
    c = torch.zeros(4, dtype=torch.int32, device="cuda")
    o = torch.zeros(4, dtype=torch.float32, device="cuda")
    for width, nbins in ((0.1, 0), (0.1, 8193), (0.0, 16), (-1.0, 16)):
        with pytest.raises(mdlg.MDError):
            mdlg.disp_hist(c, o, o, c, o, o, 10, 1.0, width, nbins)


@pytest.mark.parametrize("mu2,lam,width,nbins", [(0.16, 0.0, 0.05, 64), (1.0, 0.5, 0.1, 128),
                                                 (4.0, 3.0, 0.25, 256), (0.3, 60.0, 0.02, 512),
                                                 (2.0, 1.0, 1.0, 7)])
def test_pdf_models_match_oracle(mdlg, orc, mu2, lam, width, nbins):
    pg, pw = mdlg.disp_pdf_models(mu2, lam, width, nbins)
    torch.cuda.synchronize()
    assert np.max(np.abs(pg.cpu().numpy() - orc.pdf_gauss_bins(mu2, width, nbins))) < 1e-12
    assert np.max(np.abs(pw.cpu().numpy() - orc.pdf_wsg_bins(mu2, lam, width, nbins))) < 1e-12


def test_kl_terms_match_oracle(mdlg, orc):
    rng = np.random.default_rng(5)
    R = rng.random(333); R /= R.sum(); R[[3, 40]] = 0.0
    Q = rng.random(333); Q /= Q.sum()
    K = mdlg.kl_terms(_dev(R), _dev(Q)).cpu().numpy()
    ref = orc.kl_terms(R, Q)
    assert np.allclose(K, ref, rtol=1e-14, atol=1e-300)
    assert K[3] == 0.0 and K[40] == 0.0


def test_wsg_describes_md_displacements_better_than_gaussian(mdlg, orc):
    # Fig. 2: dilute LJ gas (phi = 0.0784, T = 20) over the paper's Delta t =
    # 3.2: the measured displacement PDF is closer, in D_KL, to the Poisson
    # WSG at the measured mu2 and mu4 than to the Gaussian of the same second
    # moment.  (Measured: kurtosis 3.18, D_KL 4e-5 against 6e-4 with 64 bins;
    # the sampling floor of D_KL is about (bins - 1) / (2 samples) = 6e-5.)
    n, phi, T = 262144, 0.0784, 20.0
    L = inputs.box_length(n, phi)
    st = inputs.lattice_gas_state(n, L, T, seed=77)
    p = mdlg.make_params(n, L, dt=5e-4, precision=mdlg.MD_FP32_CELLOFF, W=4, lg_every=(400,),
                         lx=(int(round(L)),))
    s = mdlg.System(p, st.x, st.y, st.vx, st.vy)
    s.step(4000)                                # relax the lattice start
    info = s.rep_info(0)
    a = [t.clone() for t in s.get_raw()]
    s.step(6400)                                # Delta t = 3.2
    b = s.get_raw()
    s.sync()
    nc, h = int(info.ncell), float(info.h)
    _, _, mom = mdlg.mdlg_bin(a[0], a[1], a[2], b[0], b[1], b[2], nc, h, 101, 4)
    m = mom.cpu().numpy()
    mu2, mu4 = m[0] / (2 * n), m[1] / (2 * n)
    assert 3.0 < mu4 / mu2 ** 2 < 3.75          # inside the WSG domain
    lam_t, rc = mdlg.wsg_lambda(mu2, mu4)
    lam = float(lam_t.item())
    width = 0.25 * math.sqrt(mu2)
    nbins = 64
    hist, out = mdlg.disp_hist(a[0], a[1], a[2], b[0], b[1], b[2], nc, h, width, nbins)
    R = hist.double() / (2 * n)
    pg, pw = mdlg.disp_pdf_models(mu2, lam, width, nbins)
    kg = mdlg.kl_terms(R, pg).sum().item()
    kw = mdlg.kl_terms(R, pw).sum().item()
    assert int(out.item()) < 2 * n * 1e-3
    assert kw < 0.25 * kg, (kw, kg)
    s.close()
