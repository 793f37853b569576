"""Pins of the oracle's block bootstrap of the measured equilibrium
(or_bootstrap_feq) and of its draws (SplitMix64 as a counter-based
generator), against what the definition fixes:
  * blocks that all hold the same counts give sigma = 0 (up to the rounding
    of the mean of identical values);
  * with equal windows per block, the bootstrap variance of a mean of u
    blocks tends to the population variance of the block values over u,
    sum (x_b - mean)^2 / u^2;
  * with two blocks of unequal windows the four equally likely resamples
    are known: the bootstrap standard deviation tends to theirs;
  * symmetric-set averaging of identical set members changes nothing;
  * the block indices drawn are uniform and consecutive draws uncorrelated;
  * the draws of seed 0 are the published first outputs of SplitMix64 from
    state 0 (tests/golden/splitmix64_state0.txt).
"""

import numpy as np
import pytest


def test_identical_blocks_give_zero(orc):
    h = np.tile(np.arange(81, dtype=np.int64) * 3 + 1, (32, 1))
    s = orc.bootstrap_feq(h, np.full(32, 2, np.int64), 4, 500.0, B=50, seed=9)
    P = h[0] / (500.0 * 2)
    assert np.all(s <= 1e-14 * P)


def test_converges_to_variance_of_the_block_mean(orc):
    rng = np.random.default_rng(1)
    u, n = 24, 1000.0
    h = np.zeros((32, 81), np.int64)
    h[:u] = rng.integers(0, 800, (u, 81))
    w = np.zeros(32, np.int64)
    w[:u] = 1                                     # 8 blocks hold no windows: never drawn
    s = orc.bootstrap_feq(h, w, 4, n, B=40_000, seed=3)
    x = h[:u] / n
    exact = np.sqrt(((x - x.mean(0)) ** 2).sum(0) / u ** 2)
    assert np.all(np.abs(s / exact - 1.0) < 0.03), np.max(np.abs(s / exact - 1.0))


def test_two_unequal_blocks(orc):
    n = 100.0
    h = np.zeros((32, 81), np.int64)
    h[0, 40], h[1, 40] = 30, 170                 # block 0: 1 window, block 1: 3 windows
    w = np.zeros(32, np.int64)
    w[0], w[1] = 1, 3
    s = orc.bootstrap_feq(h, w, 4, n, B=40_000, seed=5)
    # resamples (0,0), (0,1), (1,0), (1,1), each with probability 1/4
    P = np.array([60 / (n * 2), 200 / (n * 4), 200 / (n * 4), 340 / (n * 6)])
    exact = np.sqrt(np.mean((P - P.mean()) ** 2))
    assert abs(s[40] / exact - 1.0) < 0.03
    assert s[0] == 0.0


def test_symmetrize_of_identical_members(orc):
    rng = np.random.default_rng(2)
    W, side = 4, 9
    base = rng.integers(0, 500, (32, 15))
    h = np.zeros((32, 81), np.int64)
    keys = {}
    for i in range(81):
        a, b = abs(i % side - W), abs(i // side - W)
        k = (min(a, b), max(a, b))
        keys.setdefault(k, len(keys))
        h[:, i] = base[:, keys[k]]
    w = np.ones(32, np.int64)
    a = orc.bootstrap_feq(h, w, W, 700.0, sym=False, B=300, seed=7)
    b = orc.bootstrap_feq(h, w, W, 700.0, sym=True, B=300, seed=7)
    assert np.allclose(a, b, rtol=1e-14, atol=0)


def test_draws_uniform_and_uncorrelated(orc):
    from scipy import stats

    c = np.arange(200_000, dtype=np.uint64)
    x = np.array([orc.splitmix64(12345, int(v)) for v in c[:200_000:4]], dtype=np.uint64)
    idx = ((x >> np.uint64(32)) * np.uint64(32)) >> np.uint64(32)
    counts = np.bincount(idx.astype(np.int64), minlength=32)
    chi2 = float(((counts - counts.mean()) ** 2 / counts.mean()).sum())
    assert stats.chi2.sf(chi2, 31) > 1e-3
    u = (x >> np.uint64(11)).astype(np.float64) / 2.0 ** 53
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) < 5.0 / np.sqrt(len(u))


def test_draws_match_published_splitmix64(orc):
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_state0.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for c, v in rows:
        assert orc.splitmix64(0, int(c)) == int(v, 16), (c, v)
