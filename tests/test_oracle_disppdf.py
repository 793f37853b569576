"""Pins of the oracle's displacement-PDF diagnostics (Sec. 3(b), Fig. 2):
the histogram of the continuous per-axis displacement over bins X_i, the bin
masses of the Gaussian (Eq. gaussian_df) and Poisson WSG (Eqs. poisson_v2,
p_wsg_one) displacement PDFs, and the element-wise K(X_i) of Eq. k_Xi."""

import math

import numpy as np
import pytest


def _simpson(f, a, b, m=400):
    x = np.linspace(a, b, 2 * m + 1)
    y = f(x)
    return (b - a) / (6 * m) * (y[0] + y[-1] + 4 * y[1:-1:2].sum() + 2 * y[2:-1:2].sum())


@pytest.mark.parametrize("mu2,width", [(0.16, 0.05), (1.0, 0.25), (9.0, 1.0)])
def test_gaussian_bins_are_integrals_of_the_pdf(orc, mu2, width):
    nb = 64
    P = orc.pdf_gauss_bins(mu2, width, nb)
    pdf = lambda x: np.exp(-x * x / (2 * mu2)) / math.sqrt(2 * math.pi * mu2)
    for k in (0, 5, nb // 2 - 1, nb // 2, nb - 1):
        a = (k - nb // 2) * width
        assert abs(P[k] - _simpson(pdf, a, a + width)) < 1e-12
    assert np.allclose(P[: nb // 2], P[nb // 2:][::-1], rtol=0, atol=1e-15)      # symmetry


@pytest.mark.parametrize("lam", [0.2, 1.0, 3.0])
def test_wsg_bins_are_integrals_of_the_mixture(orc, lam):
    mu2, width, nb = 0.8, 0.1, 80
    P = orc.pdf_wsg_bins(mu2, lam, width, nb)
    w = lambda c: math.exp(-lam) * lam ** c / math.factorial(c)
    def pdf(x):
        s = np.zeros_like(x)
        for c in range(60):
            var = (c + 1) * mu2 / (lam + 1)
            s += w(c) * np.exp(-x * x / (2 * var)) / math.sqrt(2 * math.pi * var)
        return s
    for k in (3, nb // 2 - 1, nb // 2 + 7):
        a = (k - nb // 2) * width
        assert abs(P[k] - _simpson(pdf, a, a + width)) < 1e-12


def test_wsg_at_lambda_zero_is_gaussian(orc):
    assert np.allclose(orc.pdf_wsg_bins(0.5, 0.0, 0.1, 50), orc.pdf_gauss_bins(0.5, 0.1, 50),
                       rtol=0, atol=1e-16)


@pytest.mark.parametrize("lam", [0.0, 0.5, 2.0])
def test_grouped_moments_follow_sheppard(orc, lam):
    # fine bins covering the mass: grouped moments = continuous ones plus
    # Sheppard's corrections; the continuous ones are mu2 and Eq. fourth_order
    mu2, width = 1.0, 0.01
    nb = int(2 * 40 / width)
    P = orc.pdf_wsg_bins(mu2, lam, width, nb)
    m = (np.arange(nb) - nb // 2 + 0.5) * width
    assert abs(P.sum() - 1.0) < 1e-12
    m2 = (P * m ** 2).sum()
    m4 = (P * m ** 4).sum()
    mu4 = 3 * mu2 ** 2 * (lam ** 2 + 3 * lam + 1) / (lam + 1) ** 2
    assert abs(m2 - (mu2 + width ** 2 / 12)) < 1e-9
    assert abs(m4 - (mu4 + mu2 * width ** 2 / 2 + 7 * width ** 4 / 240)) < 1e-8


def _snap(pairs, ncell, h):
    """Hand-made snapshot pair from (x0, y0, x1, y1) absolute positions."""
    def enc(x, y):
        cx, cy = int(x // h), int(y // h)
        return cy * ncell + cx, x - cx * h, y - cy * h
    s = {k: [] for k in ("cell0", "ox0", "oy0", "cell1", "ox1", "oy1")}
    for x0, y0, x1, y1 in pairs:
        for t, (x, y) in (("0", (x0, y0)), ("1", (x1, y1))):
            c, ox, oy = enc(x, y)
            s["cell" + t].append(c)
            s["ox" + t].append(ox)
            s["oy" + t].append(oy)
    return {k: np.array(v, dtype=np.int32 if k.startswith("cell") else np.float64)
            for k, v in s.items()}


def test_hand_counted_histogram(orc):
    ncell, h = 8, 2.0          # L = 16, exact in binary
    L = ncell * h
    # displacements (dx, dy): 0.25 (bin edge: upper bin), -0.25, wrap 15.5 -> -0.5,
    # 0.75, and 3.0 (outside 8 bins of width 0.25 -> [-1, 1))
    pairs = [(1.0, 1.0, 1.25, 0.75), (15.75, 3.0, 0.25, 3.75), (4.0, 4.0, 7.0, 4.0)]
    s = _snap(pairs, ncell, h)
    hist, out = orc.disp_hist(s, ncell, h, L, 0.25, 8)
    want = np.zeros(8, np.int64)
    for d in (0.25, -0.25, 0.5, 0.75, 0.0):
        want[int(math.floor(d / 0.25)) + 4] += 1
    assert out == 1                            # the 3.0 displacement
    assert np.array_equal(hist, want)
    assert hist.sum() + out == 2 * len(pairs)


def test_kl_terms_sum_to_kl(orc):
    rng = np.random.default_rng(3)
    R = rng.random(40); R /= R.sum()
    Q = rng.random(40); Q /= Q.sum()
    R[7] = 0.0
    K = orc.kl_terms(R, Q)
    assert K[7] == 0.0
    assert abs(K.sum() - orc.kl(R, Q)) < 1e-15
    assert orc.kl(R / R.sum(), Q) >= 0.0
    assert np.allclose(orc.kl_terms(Q, Q), 0.0, atol=0)
