"""Host logic of the surrogate's fallback routing (no GPU): the trusted
region is the training box intersected with the per-phi range of training
temperatures, so queries in a corner of the box that no training replica
reached go to the WSG fallback."""

import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2101_01160_gb300 import surrogate  # noqa: E402


def _set(X):
    n = len(X)
    z = np.zeros((n, 81))
    return surrogate.DataSet(np.asarray(X, np.float32), z.astype(np.float32), z, z, np.arange(n),
                             np.ones(n), np.zeros((n, 3)))


def test_envelope_follows_the_training_support():
    rng = np.random.Generator(np.random.PCG64(3))
    phi = rng.uniform(0.02, 0.30, 4000)
    # support shaped like the relaxed MD ensemble: the lowest temperature
    # rises with density, the highest falls
    T = rng.uniform(1.0 + 5.0 * phi, 20.0 - 3.0 * phi)
    X = np.stack([phi, T, np.full_like(phi, 0.1), np.full_like(phi, 2.0)], 1)
    ds = _set(X)
    edges, t_lo, t_hi = surrogate.Predictor.envelope_of(ds, bins=14)
    assert len(edges) == 15 and np.all(np.isfinite(t_lo)) and np.all(np.isfinite(t_hi))
    assert np.all(t_lo[1:] >= t_lo[:-1] - 0.2)           # rises with phi, up to sampling
    # every training input is trusted
    pred = surrogate.Predictor([], *surrogate.Predictor.box_of(ds), envelope=(edges, t_lo, t_hi))
    assert pred.trusted(X).all()
    q = np.array([[0.25, 1.5, 0.1, 2.0],     # cold and dense: inside the box, below the support
                  [0.25, 8.0, 0.1, 2.0],     # inside the support
                  [0.03, 1.6, 0.1, 2.0],     # cold and dilute: inside the support
                  [0.25, 19.6, 0.1, 2.0],    # hot and dense: above the support
                  [0.40, 8.0, 0.1, 2.0],     # phi outside the box
                  [0.25, 8.0, 0.3, 2.0]],    # interval outside the box
                 np.float32)
    assert list(pred.trusted(q)) == [False, True, True, False, False, False]
    # without an envelope only the box decides
    box_only = surrogate.Predictor([], *surrogate.Predictor.box_of(ds))
    assert list(box_only.trusted(q)) == [True, True, True, True, False, False]


def test_empty_envelope_bin_trusts_nothing():
    X = np.array([[0.02, 5.0, 0.1, 2.0], [0.03, 6.0, 0.1, 2.0], [0.30, 5.0, 0.1, 2.0]])
    ds = _set(X)
    env = surrogate.Predictor.envelope_of(ds, bins=4)
    assert np.isinf(env[1][1]) and np.isinf(env[1][2])    # no input in the middle bins
    pred = surrogate.Predictor([], *surrogate.Predictor.box_of(ds), envelope=env)
    assert list(pred.trusted(np.array([[0.15, 5.0, 0.1, 2.0], [0.025, 5.5, 0.1, 2.0]], np.float32))) == [False, True]
