"""Pins of the surrogate oracle (oracle/mlp_oracle.c): the forward pass is a
probability distribution, the loss is the KL divergence of Eq.
(kullback_leibler) computed independently here, and the gradient equals a
central finite difference of the loss for every parameter tensor."""

import numpy as np


def _net(rng, sizes):
    Ws = [rng.normal(0, 1 / np.sqrt(a), (b, a)) for a, b in zip(sizes[:-1], sizes[1:])]
    bs = [rng.normal(0, 0.1, b) for b in sizes[1:]]
    return Ws, bs


def test_forward_is_distribution_and_loss_is_kl(orc):
    rng = np.random.default_rng(0)
    sizes = [4, 16, 16, 9]
    Ws, bs = _net(rng, sizes)
    params = orc.mlp_pack(Ws, bs)
    X = rng.uniform(-1, 1, (7, 4))
    shift, scale = np.array([0.1, 0.2, 0.0, -0.1]), np.array([1.0, 2.0, 0.5, 1.5])
    P = orc.mlp_forward(sizes, X, params, shift, scale)
    assert np.allclose(P.sum(1), 1.0, atol=1e-14) and np.all(P > 0)
    # an independent numpy forward pass
    h = (X - shift) / scale
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = h @ W.T + b
        h = z / (1 + np.exp(-z)) if l < len(Ws) - 1 else z
    ref = np.exp(h - h.max(1, keepdims=True))
    ref /= ref.sum(1, keepdims=True)
    assert np.max(np.abs(P - ref)) < 1e-14
    T = rng.dirichlet(np.ones(9), 7)
    loss, _ = orc.mlp_loss_backward(sizes, X, params, T, shift, scale)
    assert abs(loss - np.mean(np.sum(T * np.log(T / P), 1))) < 1e-14


def test_gradient_matches_finite_differences(orc):
    rng = np.random.default_rng(1)
    sizes = [4, 12, 10, 7]
    Ws, bs = _net(rng, sizes)
    params = orc.mlp_pack(Ws, bs)
    X = rng.uniform(-1, 1, (5, 4))
    T = rng.dirichlet(np.ones(7), 5)
    T[0, 3] = 0.0            # zero target entries take the 0 log 0 = 0 branch
    T[0] /= T[0].sum()
    shift, scale = np.zeros(4), np.ones(4)
    loss, g = orc.mlp_loss_backward(sizes, X, params, T, shift, scale)
    eps = 1e-6
    idx = np.concatenate([rng.choice(len(params), 60, replace=False), [0, len(params) - 1]])
    for i in idx:
        pp = params.copy(); pp[i] += eps
        pm = params.copy(); pm[i] -= eps
        lp, _ = orc.mlp_loss_backward(sizes, X, pp, T, shift, scale)
        lm, _ = orc.mlp_loss_backward(sizes, X, pm, T, shift, scale)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])
