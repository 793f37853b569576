"""GPU parity of the surrogate's tensor-core kernels: the tcgen05 BF16 GEMM
against an FP32 product of the same BF16 operands, the MLP forward pass and
its gradient against the FP64 oracle (oracle/mlp_oracle.c), and a training
run that lowers the loss."""

import numpy as np
import pytest

from paper_2101_01160_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHIFT = np.array([0.16, 10.5, 0.5, 1.25])
SCALE = np.array([0.14, 9.5, 0.5, 0.75])


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (128, 256, 256), (256, 96, 128),
                                   (1024, 128, 1024), (384, 256, 192)])
def test_tcgen05_gemm(mdlg, M, N, K):
    g = torch.Generator(device="cpu").manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C, st = mdlg.bf16_gemm_tn(A, B)
    torch.cuda.synchronize()
    assert st.item() == 0
    ref = A.float() @ B.float().T
    err = (C - ref).abs().max().item()
    assert err <= 1e-4 * ref.abs().max().item() + 1e-5, err


def _model(mdlg, seed=0):
    Ws, bs = inputs.mlp_init(mdlg.SURR_SIZES, seed)
    from oracle import oracle

    params = oracle.mlp_pack(Ws, bs).astype(np.float32)
    return mdlg.MLP(params, SHIFT, SCALE), params


def _queries(n, seed):
    return inputs.surrogate_queries(n, seed)


def test_forward_matches_oracle(mdlg, orc):
    m, params = _model(mdlg)
    X = _queries(300, 1)
    P = m.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    m.status()
    ref = orc.mlp_forward(mdlg.SURR_SIZES, X.astype(np.float64), params.astype(np.float64), SHIFT, SCALE)
    assert np.allclose(P.sum(1), 1.0, atol=1e-5)
    # BF16 weights and activations against FP64: relative 3e-2 on every class
    assert np.max(np.abs(P - ref) / (ref + 1e-4)) < 3e-2, np.max(np.abs(P - ref))


def test_gradient_matches_oracle(mdlg, orc):
    m, params = _model(mdlg, seed=1)
    B = 256
    X = _queries(B, 2)
    rng = np.random.default_rng(3)
    T = rng.dirichlet(np.ones(81) * 0.5, B).astype(np.float32)
    g, loss = m.grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    m.status()
    g = g.cpu().numpy().astype(np.float64)
    lref, gref = orc.mlp_loss_backward(mdlg.SURR_SIZES, X.astype(np.float64), params.astype(np.float64),
                                       T.astype(np.float64), SHIFT, SCALE)
    assert abs(loss.item() - lref) < 1e-2 * abs(lref)
    off = 0
    sizes = mdlg.SURR_SIZES
    for a, b in zip(sizes[:-1], sizes[1:]):
        for n in (a * b, b):
            u, v = g[off:off + n], gref[off:off + n]
            cos = u @ v / (np.linalg.norm(u) * np.linalg.norm(v) + 1e-300)
            rel = np.linalg.norm(u - v) / (np.linalg.norm(v) + 1e-300)
            assert cos >= 0.999 and rel <= 2e-2, (off, n, cos, rel)
            off += n


def test_training_lowers_loss(mdlg, orc):
    """Fits the Gaussian equilibrium of the ballistic a^2 = T dt^2 / dx^2 (a
    smooth target family) with 1500 Adam steps."""
    m, _ = _model(mdlg, seed=2)
    rng = np.random.default_rng(4)
    N = 4096
    X = _queries(N, 5)
    a2 = X[:, 1] * X[:, 2] ** 2 / X[:, 3] ** 2 * 0.5
    T = np.stack([orc.feq_gaussian(float(max(a, 1e-3)), 0, 0, 4) for a in a2]).astype(np.float32)
    T /= T.sum(1, keepdims=True)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    loss = torch.zeros(1, device="cuda")
    losses = []
    for it in range(1500):
        idx = torch.from_numpy(rng.integers(0, N, 512)).cuda()
        m.train_step(Xd[idx].contiguous(), Td[idx].contiguous(), 2e-3 if it < 1000 else 5e-4,
                     loss=loss)
        if it % 100 == 0 or it == 1499:
            losses.append(loss.item())
    m.status()
    assert losses[-1] < 0.2 * losses[0], losses
    P = m.forward(Xd).cpu().numpy()
    assert np.max(np.abs(P - T)) < 0.05


def test_surrogate_pipeline_beats_md_free_baseline(mdlg):
    """End to end on a reduced ensemble: MD-measured equilibria as training
    data, tensor-core training, held-out replicas run 5x longer (their
    labels' sampling error is small against the bar); the surrogate (no MD
    at query time) must beat the ballistic Gaussian (the other MD-free
    prediction) and stay within 1.5e-2 of every measured class (measured
    9.1e-3 with this small set and short training; the full pipeline of
    surrogate.main reaches 1.4e-3 with one network, 1.05e-3 with its
    four-network predictor)."""
    from paper_2101_01160_gb300 import surrogate

    tr = surrogate.generate(31, n_rep=96, steps=8000, n_equil=2000, n_min=2048, n_max=8192)
    te = surrogate.generate(32, n_rep=24, steps=40_000, n_equil=2000, n_min=2048, n_max=8192,
                            rep_offset=5000)
    assert len(tr.X) > 300 and len(te.X) > 60
    m = surrogate.new_model(3)
    hist = surrogate.train(m, tr, steps=6000, lr=1e-3, batch=512, log_every=1000)
    assert hist[-1][1] < 0.3 * hist[0][1], hist
    res = surrogate.evaluate(m, te)
    print(res)
    assert res["surrogate"]["median"] < res["gauss_ballistic"]["median"], res
    assert res["surrogate"]["max"] < 1.5e-2, res


def test_predictor_falls_back_to_wsg(mdlg):
    """Outside the training box, or where the two networks disagree beyond
    the tolerance, the prediction is the WSG equilibrium at the supplied
    moments (Eqs. f_eq_wsg, lambda_eq); inside, the networks' mean."""
    import torch

    from paper_2101_01160_gb300 import surrogate

    ms = [surrogate.new_model(s) for s in (5, 6)]
    lo, hi = np.array([0.02, 1.0, 0.05, 1.0]), np.array([0.30, 20.0, 0.2, 4.0])
    X = np.array([[0.1, 10.0, 0.1, 2.0],      # inside
                  [0.5, 10.0, 0.1, 2.0],      # phi outside
                  [0.1, 30.0, 0.1, 2.0]], np.float32)
    mom = np.array([[0.05, 0.05 ** 2 * 3.3, 1.0], [0.3, 0.3 ** 2 * 3.2, 2.0], [0.9, 0.9 ** 2 * 3.1, 2.0]])
    pred = surrogate.Predictor(ms, lo, hi, tol=1.0)      # no disagreement limit
    P, fb, spread = pred(X, mom)
    assert list(fb) == [False, True, True]
    mean = np.mean([m.forward(torch.from_numpy(X).cuda()).cpu().numpy() for m in ms], axis=0)
    assert np.allclose(P[0], mean[0], rtol=0, atol=1e-7)
    for i in (1, 2):
        mu2, mu4, dx = mom[i]
        lam, _ = mdlg.wsg_lambda(mu2, mu4, allow_domain=True)
        ref = mdlg.feq_wsg(mu2 / dx ** 2, lam.item(), W=4).cpu().numpy()
        assert np.array_equal(P[i], ref)
    # untrained networks of different seeds disagree: a tight limit sends
    # every query to the fallback
    P2, fb2, sp2 = surrogate.Predictor(ms, lo, hi, tol=1e-6)(X, mom)
    assert fb2.all() and np.all(sp2 > 1e-6)
    with pytest.raises(ValueError):
        pred(X)
