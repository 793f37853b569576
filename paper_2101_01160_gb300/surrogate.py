"""Training and evaluation pipeline of the f_eq surrogate (a project addition,
not in the paper), driving the library's kernels:

1. ``generate``: batched MD runs (md_init_batch / md_step) at random state
   points (phi, T) measure the equilibrium f_eq on several sampling intervals
   and lattice spacings (feq_batch); each (replica, interval, lattice) with a
   negligible overflow fraction is one labelled example
   x = (phi, T, Delta t_LG, Delta x_eff) -> measured probabilities.
2. ``train``: Adam on the mean KL divergence with the tensor-core MLP
   (mlp_train_step); minibatches are slices of a host-shuffled, device
   resident copy of the data set.
3. ``evaluate``: on held-out replicas, the largest absolute deviation from
   the measured distribution of the surrogate, of the Gaussian equilibrium at
   the ballistic a^2 = T dt^2 / dx^2 (needs no MD), and of the Gaussian and
   WSG equilibria at the measured moments (need an MD run).

Python here only sequences library calls and moves arrays.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import inputs, mdlg

SHIFT = np.array([0.16, 10.5, 0.1, 2.0])      # feature centres (phi, T, dt_lg, dx)
SCALE = np.array([0.14, 9.5, 0.1, 1.5])       # feature half-ranges


@dataclass
class DataSet:
    X: np.ndarray        # [n, 4] (phi, T, dt_lg, dx_eff)
    P: np.ndarray        # [n, 81] measured, normalised over the window
    G: np.ndarray        # [n, 81] Gaussian at the measured a^2
    Wsg: np.ndarray      # [n, 81] WSG at the measured a^2, lambda
    rep: np.ndarray      # [n] replica id (for held-out splits)
    samples: np.ndarray  # [n] particle-windows behind each histogram


def generate(seed: int, n_rep: int = 256, steps: int = 20_000, n_equil: int = 4000,
             lg_every=(100, 200, 400), dxs=(1.0, 2.0, 4.0), dt: float = 5e-4,
             max_overflow: float = 1e-4, rep_offset: int = 0, n_min=4096, n_max=65536) -> DataSet:
    import torch

    Ns, phis, Ts = inputs.ensemble_params(n_rep, seed=seed, n_min=n_min, n_max=n_max)
    params, cat = [], [[], [], [], []]
    for r in range(n_rep):
        n = int(Ns[r])
        L = inputs.box_length(n, float(phis[r]))
        st = inputs.lattice_gas_state(n, L, float(Ts[r]), seed=1_000_000 + 1000 * seed + r)
        params.append(mdlg.make_params(n, L, dt=dt, precision=mdlg.MD_FP32_CELLOFF, W=4,
                                       n_equil=n_equil, lg_every=lg_every,
                                       lx=tuple(int(round(L / d)) for d in dxs)))
        for a, f in zip(cat, ("x", "y", "vx", "vy")):
            a.append(getattr(st, f))
    s = mdlg.System(params, *[np.concatenate(a) for a in cat])
    s.autotune(50)
    s.step(n_equil + steps)
    s.sync()
    X, P, G, Wg, rep, samp = [], [], [], [], [], []
    for k, every in enumerate(lg_every):
        for d in range(len(dxs)):
            Pm, Gm, Wm, stt = mdlg.feq_batch(s, k, d, symmetrize=True)
            ovf = stt[:, 10] / np.maximum(stt[:, 9], 1.0)
            keep = (ovf <= max_overflow) & (stt[:, 9] > 0)
            for r in np.nonzero(keep)[0]:
                X.append((phis[r], Ts[r], every * dt, stt[r, 11]))
                P.append(Pm[r] / Pm[r].sum())
                G.append(Gm[r])
                Wg.append(Wm[r])
                rep.append(rep_offset + r)
                samp.append(stt[r, 9])
    s.close()
    torch.cuda.synchronize()
    return DataSet(np.array(X, np.float32), np.array(P, np.float32), np.array(G), np.array(Wg),
                   np.array(rep), np.array(samp))


def concat(sets):
    return DataSet(*[np.concatenate([getattr(s, f) for s in sets]) for f in
                     ("X", "P", "G", "Wsg", "rep", "samples")])


def split(ds: DataSet, frac: float, seed: int):
    reps = np.unique(ds.rep)
    rng = np.random.Generator(np.random.PCG64(seed))
    held = set(rng.choice(reps, max(1, int(round(frac * len(reps)))), replace=False).tolist())
    m = np.array([r in held for r in ds.rep])
    pick = lambda mask: DataSet(*[getattr(ds, f)[mask] for f in ("X", "P", "G", "Wsg", "rep", "samples")])
    return pick(~m), pick(m)


def new_model(seed: int) -> mdlg.MLP:
    Ws, bs = inputs.mlp_init(mdlg.SURR_SIZES, seed)
    params = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in zip(Ws, bs)])
    return mdlg.MLP(params, SHIFT, SCALE)


def train(model: mdlg.MLP, ds: DataSet, steps: int = 6000, batch: int = 512, lr: float = 2e-3,
          seed: int = 0, log_every: int = 0):
    """Adam with a cosine learning-rate decay; returns the loss history."""
    import torch

    n = len(ds.X)
    reps = max(1, math.ceil(batch / n))          # small sets: repeat rows to fill a batch
    rng = np.random.Generator(np.random.PCG64(seed))
    Xd = torch.from_numpy(np.tile(ds.X, (reps, 1))).cuda()
    Pd = torch.from_numpy(np.tile(ds.P, (reps, 1))).cuda()
    n_all = Xd.shape[0]
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    order = torch.from_numpy(rng.permutation(n_all)).cuda()
    Xs, Ps = Xd[order].contiguous(), Pd[order].contiguous()
    pos = 0
    for it in range(steps):
        if pos + batch > n_all:
            order = torch.from_numpy(rng.permutation(n_all)).cuda()
            Xs, Ps = Xd[order].contiguous(), Pd[order].contiguous()
            pos = 0
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * it / steps))
        model.train_step(Xs[pos:pos + batch], Ps[pos:pos + batch], lr_t, loss=loss)
        pos += batch
        if log_every and (it % log_every == 0 or it == steps - 1):
            hist.append((it, loss.item()))
    model.status()
    return hist


def evaluate(model: mdlg.MLP, ds: DataSet) -> dict:
    """Largest absolute deviation per example from the measured distribution,
    summarised over the set, for the surrogate and the analytic equilibria."""
    import torch

    P = model.forward(torch.from_numpy(ds.X).cuda()).cpu().numpy()
    ballistic = []
    for x in ds.X:
        a2 = float(x[1]) * float(x[2]) ** 2 / float(x[3]) ** 2
        ballistic.append(mdlg.feq_gaussian(a2, W=4).cpu().numpy())
    ballistic = np.array(ballistic)

    def summary(Q):
        e = np.max(np.abs(Q - ds.P), axis=1)
        return {"max": float(e.max()), "median": float(np.median(e)), "mean": float(e.mean())}

    # statistical floor: one standard error of the largest class
    floor = np.sqrt(ds.P.max(1) * (1 - ds.P.max(1)) / ds.samples)
    return {"surrogate": summary(P), "gauss_ballistic": summary(ballistic),
            "gauss_measured_a2": summary(ds.G), "wsg_measured": summary(ds.Wsg),
            "sampling_sigma_median": float(np.median(floor)), "n": int(len(ds.X))}


def inference_throughput(model: mdlg.MLP, n: int = 1 << 20, reps: int = 5, seed: int = 0) -> dict:
    """Device time of model.forward on n query points (after one warm call)."""
    import torch

    # uniform in the training box: phi, T, dt_lg, dx
    X = torch.from_numpy(inputs.surrogate_queries(n, seed, lo=(0.02, 1.0, 0.05, 1.0),
                                                  hi=(0.30, 20.0, 0.2, 4.0))).cuda()
    out = torch.empty((n, model.n_classes), dtype=torch.float32, device="cuda")
    model.forward(X, out=out)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        model.forward(X, out=out)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    model.status()
    ms = float(np.median(ts))
    sizes = mdlg.SURR_SIZES
    flop = 2.0 * sum(a * b for a, b in zip(sizes[:-1], sizes[1:])) * n
    return {"queries": n, "ms": ms, "queries_per_s": n / (ms * 1e-3), "tflops": flop / (ms * 1e-3) / 1e12,
            "flop_per_query": flop / n}


def main():
    import json
    import time

    t0 = time.time()
    sets = [generate(seed, rep_offset=1000 * seed) for seed in (21, 22, 23, 24)]
    ds = concat(sets)
    tr, te = split(ds, 0.1, seed=5)
    t1 = time.time()
    model = new_model(0)
    hist = train(model, tr, steps=8000, log_every=1000)
    t2 = time.time()
    res = {"train_examples": len(tr.X), "test_examples": len(te.X), "md_seconds": t1 - t0,
           "train_seconds": t2 - t1, "loss": hist, "test": evaluate(model, te),
           "train": evaluate(model, tr), "inference": inference_throughput(model)}
    print(json.dumps(res))


if __name__ == "__main__":
    main()
