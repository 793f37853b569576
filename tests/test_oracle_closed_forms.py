"""Pins of the oracle's closed forms (Sec. 3) against things the paper and the
mathematics fix independently of the oracle's own code:

* the defining integral of f^eq (Eq. theory_feq) evaluated by numerical
  quadrature with scipy, for the single Gaussian (Eq. gaussian_df) and for the
  Poisson mixture of Gaussians (Eqs. poisson_v2, p_wsg_one);
* normalisation and first moment of the lattice distribution;
* WSG with lambda = 0 reduces to the single Gaussian (Sec. 1);
* the continuous mixture's fourth moment (Eq. fourth_order), by quadrature;
* the roots of Eq. (lambda_eq): lambda1*lambda2 = 1, the closed form at
  kurtosis 3.6, the double root at 3.75, and the residual of the quadratic;
* the Poisson truncation tail against scipy's survival function;
* KL divergence (Eq. kullback_leibler) against scipy.stats.entropy;
* symmetric-set averaging (Sec. 5) against the average over the 8 symmetries
  of the square.
"""

import math

import numpy as np
import pytest
from scipy import integrate, stats

A2S = [1.0 / 6.0, 0.1611, 0.05, 0.8, 3.0]


def _tri_conv(v, var, mean=0.0):
    """P(v) = int ds g(s) tri(s - v): a particle uniform in a unit cell that is
    displaced by s ~ N(mean, var) lands v cells away (Eq. theory_feq in 1D)."""
    sd = math.sqrt(var)
    f = lambda s: stats.norm.pdf(s, mean, sd) * (1.0 - abs(s - v))
    a, b = integrate.quad(f, v - 1.0, v, epsabs=1e-15, epsrel=1e-13)[0], \
        integrate.quad(f, v, v + 1.0, epsabs=1e-15, epsrel=1e-13)[0]
    return a + b


def _cell_integral(v, var, mean=0.0):
    """The same probability straight from the definition: start x0 uniform in
    [0,1), displaced by s; count it in class v if floor(x0 + s) == v."""
    sd = math.sqrt(var)
    # for fixed x0 the s-range landing in cell v is [v - x0, v + 1 - x0)
    g = lambda x0: stats.norm.cdf(v + 1 - x0, mean, sd) - stats.norm.cdf(v - x0, mean, sd)
    return integrate.quad(g, 0.0, 1.0, epsabs=1e-15, epsrel=1e-13)[0]


@pytest.mark.parametrize("a2", A2S)
def test_gaussian_1d_matches_defining_integral(orc, a2):
    for v in range(-4, 5):
        for u in (0.0, 0.3, -0.45):
            ref = _tri_conv(v, a2, mean=u)
            got = orc.feq_g1(v - u, a2)
            assert abs(got - ref) < 2e-13, (v, u, got, ref)


def test_triangle_form_equals_cell_definition():
    # ties the quadrature used above to the plain definition once
    for a2 in (0.1611, 0.8):
        for v in (-2, 0, 1, 3):
            assert abs(_tri_conv(v, a2) - _cell_integral(v, a2)) < 1e-12


@pytest.mark.parametrize("a2", A2S)
def test_gaussian_normalisation_and_mean(orc, a2):
    W = 40
    for u in (0.0, 0.25, -0.7):
        P = orc.feq_gaussian(a2, u, -u, W).reshape(2 * W + 1, 2 * W + 1)
        v = np.arange(-W, W + 1)
        assert abs(P.sum() - 1.0) < 1e-13
        assert abs((P.sum(axis=0) * v).sum() - u) < 1e-12
        assert abs((P.sum(axis=1) * v).sum() + u) < 1e-12


def test_d2q9_weights_at_a2_one_sixth(orc):
    # Sec. 3(a): at a^2 ~ 1/6 the Gaussian equilibrium approximates the D2Q9
    # lattice Boltzmann weights 4/9, 1/9, 1/36 (approximately, not exactly).
    P = orc.feq_gaussian(1.0 / 6.0, 0.0, 0.0, 1).reshape(3, 3)
    assert abs(P[1, 1] - 4 / 9) < 0.015
    assert abs(P[1, 2] - 1 / 9) < 0.005
    assert abs(P[2, 2] - 1 / 36) < 0.003
    # and the values computed by quadrature of the definition
    assert abs(P[1, 1] - _tri_conv(0, 1 / 6) ** 2) < 1e-13


def _mixture_weights(lam):
    cmax = int(math.ceil(lam + 12 * math.sqrt(lam) + 20)) if lam > 0 else 0
    c = np.arange(cmax + 1)
    return c, stats.poisson.pmf(c, lam) if lam > 0 else np.array([1.0])


@pytest.mark.parametrize("a2,lam", [(0.1611, 0.5), (0.1611, 2.618), (0.8, 1.2), (0.05, 7.0)])
def test_wsg_matches_defining_integral(orc, a2, lam):
    """f_i = sum_c Pois(c) prod_alpha F_c(v_alpha), F_c the 1D cell integral of
    a Gaussian of variance a^2 (c+1)/(lambda+1) (Eq. p_wsg_one, d = 1)."""
    W = 3
    c, w = _mixture_weights(lam)
    F = np.array([[_tri_conv(v, a2 * (cc + 1) / (lam + 1)) for v in range(-W, W + 1)]
                  for cc in c[w > 1e-18]])
    ww = w[w > 1e-18]
    ref = np.einsum("c,ci,cj->ij", ww, F, F).ravel()   # [vy][vx]
    got = orc.feq_wsg(a2, lam, 0.0, 0.0, W)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_wsg_lambda_zero_is_gaussian(orc):
    for a2 in A2S:
        for u in (0.0, 0.2):
            g = orc.feq_gaussian(a2, u, 0.1, 4)
            w = orc.feq_wsg(a2, 0.0, u, 0.1, 4)
            assert np.max(np.abs(g - w)) < 1e-15


@pytest.mark.parametrize("mu2,lam", [(1.0, 0.3), (0.4, 2.618), (2.0, 10.0)])
def test_fourth_moment_of_mixture(orc, mu2, lam):
    c, w = _mixture_weights(lam)
    var = mu2 * (c + 1) / (lam + 1)
    m2 = float(np.sum(w * var))
    m4 = float(np.sum(w * 3 * var * var))       # Gaussian 4th moment, mixed
    assert abs(m2 - mu2) < 1e-12 * mu2
    assert abs(orc.wsg_mu4(mu2, lam) - m4) < 1e-12 * m4
    # and by quadrature of the mixture density itself
    dens = lambda s: float(np.sum(w * stats.norm.pdf(s, 0, np.sqrt(var))))
    sd = math.sqrt(mu2 * (c[-1] + 1) / (lam + 1))
    q4 = integrate.quad(lambda s: s ** 4 * dens(s), -40 * sd, 40 * sd, limit=400)[0]
    assert abs(q4 - m4) < 1e-8 * m4


def test_lambda_roots(orc):
    # kurtosis 3.6: lambda^2 - 3 lambda + 1 = 0, roots (3 +- sqrt 5)/2
    rc, l1, l2 = orc.wsg_lambda(1.0, 3.6)
    assert rc == 0
    assert abs(l1 - (3 - math.sqrt(5)) / 2) < 1e-14
    assert abs(l2 - (3 + math.sqrt(5)) / 2) < 1e-14
    # kurtosis 3.75: double root lambda = 1
    rc, l1, l2 = orc.wsg_lambda(2.0, 3.75 * 4.0)
    assert rc == 0 and abs(l1 - 1) < 1e-7 and abs(l2 - 1) < 1e-7
    # outside the domain
    assert orc.wsg_lambda(1.0, 3.8)[0] == -2
    assert orc.wsg_lambda(1.0, 3.0)[0] == -1
    rng = np.random.default_rng(5)
    for _ in range(50):
        mu2 = float(rng.uniform(0.01, 5.0))
        k = float(rng.uniform(3.001, 3.749))
        mu4 = k * mu2 * mu2
        rc, l1, l2 = orc.wsg_lambda(mu2, mu4)
        assert rc == 0
        assert abs(l1 * l2 - 1.0) < 1e-9
        assert l2 >= 1.0 >= l1 > 0
        for lam in (l1, l2):
            # residual of Eq. (lambda_eq)
            res = 3 * mu2 ** 2 / (lam + 1) ** 2 * (lam ** 2 + 3 * lam + 1) - mu4
            assert abs(res) < 1e-10 * mu4
            assert abs(orc.wsg_mu4(mu2, lam) - mu4) < 1e-10 * mu4


def test_poisson_truncation_tail(orc):
    for lam in (1e-3, 0.1, 0.5, 1.0, 2.618, 10.0, 58.0, 100.0):
        cmax = orc.wsg_cmax(lam)
        assert stats.poisson.sf(cmax, lam) < 1e-16
        s = sum(orc.poisson(c, lam) for c in range(cmax + 1))
        assert abs(s - 1.0) < 1e-13
        for c in (0, 1, int(lam), cmax):
            assert abs(orc.poisson(c, lam) - stats.poisson.pmf(c, lam)) < 1e-14


def test_kl(orc):
    R = np.array([0.5, 0.5, 0.0])
    Q = np.array([0.25, 0.5, 0.25])
    assert abs(orc.kl(R, Q) - stats.entropy(R, Q)) < 1e-15
    rng = np.random.default_rng(1)
    for _ in range(10):
        a = rng.random(81)
        b = rng.random(81)
        a /= a.sum()
        b /= b.sum()
        assert abs(orc.kl(a, b) - stats.entropy(a, b)) < 1e-13
        assert orc.kl(a, a) == 0.0
        assert orc.kl(a, b) > 0.0


def test_symmetrize_is_group_average(orc):
    rng = np.random.default_rng(2)
    for W in (1, 2, 4):
        P = rng.random((2 * W + 1) ** 2)
        A = P.reshape(2 * W + 1, 2 * W + 1)
        imgs = []
        for k in range(4):
            r = np.rot90(A, k)
            imgs += [r, r.T]
        ref = np.mean(imgs, axis=0).ravel()
        got = orc.symmetrize(P, W)
        assert np.max(np.abs(got - ref)) < 1e-15
        assert abs(got.sum() - P.sum()) < 1e-13
