"""Training and evaluation pipeline of the f_eq surrogate (a project addition,
not in the paper), driving the library's kernels:

1. ``generate``: batched MD runs (md_init_batch / md_step) at random state
   points (phi, T) measure the equilibrium f_eq on several sampling intervals
   and lattice spacings (feq_batch); each (replica, interval, lattice) with a
   negligible overflow fraction is one labelled example
   x = (phi, T, Delta t_LG, Delta x_eff) -> measured probabilities, T the
   replica's kinetic temperature averaged over the sampling period.  (The
   MD is microcanonical: as the lattice start relaxes, a replica settles at
   its own temperature, up to 40 % above the initial one for the cold dense
   replicas and a few per cent below it for the hot dense ones, with a
   scatter between replicas of one state point; the initial temperature
   would make that scatter label noise.)
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
    X: np.ndarray        # [n, 4] (phi, T, dt_lg, dx_eff), T the measured kinetic temperature
    P: np.ndarray        # [n, 81] measured, normalised over the window
    G: np.ndarray        # [n, 81] Gaussian at the measured a^2
    Wsg: np.ndarray      # [n, 81] WSG at the measured a^2, lambda
    rep: np.ndarray      # [n] replica id (for held-out splits)
    samples: np.ndarray  # [n] particle-windows behind each histogram
    mom: np.ndarray      # [n, 3] measured mu2, mu4, dx_eff (the WSG fallback's inputs)


def generate(seed: int, n_rep: int = 256, steps: int = 40_000, n_equil: int = 48_000,
             lg_every=(100, 200, 400), dxs=(1.0, 2.0, 4.0), dt: float = 5e-4,
             max_overflow: float = 1e-4, rep_offset: int = 0, n_min=4096, n_max=65536,
             t_samples: int = 40) -> DataSet:
    """Labelled examples of one batched MD run (see the module docstring).
    n_equil steps relax the lattice start before sampling (the cold dense
    replicas warm for about 48,000 steps of 5e-4); the temperature feature
    averages md_energy_batch's kinetic energy at t_samples points spread
    over the sampling steps."""
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
    s.step(n_equil)
    ke, done, k_t = np.zeros(n_rep), 0, 0
    for k in range(1, t_samples + 1):
        nxt = steps * k // t_samples
        if nxt > done:
            s.step(nxt - done)
            done = nxt
            ke += s.energy_batch()[:, 0]
            k_t += 1
    if done < steps:
        s.step(steps - done)
    s.sync()
    # two dimensions, zero total momentum: KE = (2N - 2) T / 2
    T_kin = ke / max(k_t, 1) / (np.asarray(Ns, np.float64) - 1.0)
    X, P, G, Wg, rep, samp, mom = [], [], [], [], [], [], []
    for k, every in enumerate(lg_every):
        for d in range(len(dxs)):
            Pm, Gm, Wm, stt = mdlg.feq_batch(s, k, d, symmetrize=True)
            ovf = stt[:, 10] / np.maximum(stt[:, 9], 1.0)
            keep = (ovf <= max_overflow) & (stt[:, 9] > 0)
            for r in np.nonzero(keep)[0]:
                X.append((phis[r], T_kin[r], every * dt, stt[r, 11]))
                P.append(Pm[r] / Pm[r].sum())
                G.append(Gm[r])
                Wg.append(Wm[r])
                rep.append(rep_offset + r)
                samp.append(stt[r, 9])
                mom.append((stt[r, 0], stt[r, 1], stt[r, 11]))
    s.close()
    torch.cuda.synchronize()
    return DataSet(np.array(X, np.float32), np.array(P, np.float32), np.array(G), np.array(Wg),
                   np.array(rep), np.array(samp), np.array(mom))


FIELDS = ("X", "P", "G", "Wsg", "rep", "samples", "mom")


def concat(sets):
    return DataSet(*[np.concatenate([getattr(s, f) for s in sets]) for f in FIELDS])


def split(ds: DataSet, frac: float, seed: int):
    reps = np.unique(ds.rep)
    rng = np.random.Generator(np.random.PCG64(seed))
    held = set(rng.choice(reps, max(1, int(round(frac * len(reps)))), replace=False).tolist())
    m = np.array([r in held for r in ds.rep])
    pick = lambda mask: DataSet(*[getattr(ds, f)[mask] for f in FIELDS])
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


class Predictor:
    """The surrogate with the analytic WSG equilibrium (Sec. 3(b), Eqs.
    f_eq_wsg and lambda_eq) as its fallback.

    Several networks trained from different initial weights predict each
    query; their mean is the prediction where the query is trusted and the
    networks agree within `tol` in every class (the largest spread between
    them is the uncertainty estimate).  A query is trusted when it lies
    inside the box the training inputs span and, at its phi, inside the
    range of temperatures the training replicas reached (`envelope`): the
    microcanonical MD never reaches some corners of the box (dense replicas
    warm as their lattice start relaxes, so there are no cold dense
    examples), and the networks would extrapolate there.  Elsewhere the
    prediction is the WSG equilibrium at the caller's measured moments
    (mu2, mu4, dx_eff): a^2 = mu2 / dx_eff^2 and lambda from the kurtosis
    (wsg_lambda; kurtosis outside (3, 3.75] gives the Gaussian or lambda = 1
    as feq_wsg defines).  Queries that need the fallback but have no moments
    raise ValueError."""

    def __init__(self, models, lo, hi, tol=2e-3, envelope=None):
        self.models = list(models)
        self.lo = np.asarray(lo, np.float32)
        self.hi = np.asarray(hi, np.float32)
        self.tol = float(tol)
        self.envelope = envelope

    @staticmethod
    def box_of(ds: DataSet, pad=0.0):
        lo, hi = ds.X.min(0), ds.X.max(0)
        span = hi - lo
        return lo - pad * span, hi + pad * span

    @staticmethod
    def envelope_of(ds: DataSet, bins: int = 14):
        """(phi bin edges [bins + 1], lowest and highest training temperature
        per bin); an empty bin trusts no temperature."""
        X = np.asarray(ds.X, np.float64)
        edges = np.linspace(X[:, 0].min(), X[:, 0].max(), bins + 1)
        b = np.clip(np.searchsorted(edges, X[:, 0], side="right") - 1, 0, bins - 1)
        t_lo, t_hi = np.full(bins, np.inf), np.full(bins, -np.inf)
        np.minimum.at(t_lo, b, X[:, 1])
        np.maximum.at(t_hi, b, X[:, 1])
        return edges, t_lo, t_hi

    def trusted(self, X):
        """Inside the training box and, if set, the temperature envelope."""
        X = np.asarray(X, np.float32)
        ok = np.all((X >= self.lo) & (X <= self.hi), axis=1)
        if self.envelope is not None:
            edges, t_lo, t_hi = self.envelope
            b = np.clip(np.searchsorted(edges, X[:, 0].astype(np.float64), side="right") - 1, 0, len(t_lo) - 1)
            T = X[:, 1].astype(np.float64)
            ok &= (X[:, 0] >= edges[0]) & (X[:, 0] <= edges[-1]) & (T >= t_lo[b]) & (T <= t_hi[b])
        return ok

    def __call__(self, X, moments=None):
        """X float32 [n, 4]; moments float64 [n, 3] (mu2, mu4, dx_eff) or
        None.  Returns (P [n, 81] float64, fallback bool [n], spread [n])."""
        import torch

        X = np.ascontiguousarray(X, np.float32)
        Xd = torch.from_numpy(X).cuda()
        outs = np.stack([m.forward(Xd).cpu().numpy().astype(np.float64) for m in self.models])
        P = outs.mean(axis=0)
        spread = np.max(outs.max(axis=0) - outs.min(axis=0), axis=1)
        fb = ~self.trusted(X) | (spread > self.tol)
        if fb.any():
            if moments is None:
                raise ValueError("queries outside the trusted region need moments for the WSG fallback")
            mom = np.asarray(moments, np.float64)
            for i in np.nonzero(fb)[0]:
                mu2, mu4, dx = mom[i]
                lam_t, _ = mdlg.wsg_lambda(float(mu2), float(mu4), allow_domain=True)
                P[i] = mdlg.feq_wsg(float(mu2) / float(dx) ** 2, float(lam_t.item()), W=4).cpu().numpy()
        return P, fb, spread


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


def main(save=None):
    """The full pipeline: training examples from eight 256-replica MD runs
    (48,000 steps of relaxation, 80,000 of sampling), held-out examples from
    other replicas sampled 1,000,000 steps (labels with a sampling error
    well below the 1e-3 target, also for the smallest replicas), four networks trained 40,000 Adam steps from
    different initial weights, the WSG fallback where they disagree by more
    than 5e-4 or a query leaves the training box or its temperature
    envelope.  `save`: optional .npz path for the held-out inputs, labels,
    predictions and fallback flags."""
    import json
    import time

    t0 = time.time()
    tr = concat([generate(seed, rep_offset=1000 * seed, steps=80_000) for seed in range(21, 29)])
    te = concat([generate(91, n_rep=64, rep_offset=91_000, steps=1_000_000)])
    t1 = time.time()
    models = [new_model(seed) for seed in range(4)]
    hist = [train(m, tr, steps=40_000, lr=1e-3, seed=k, log_every=5000) for k, m in enumerate(models)]
    t2 = time.time()
    pred = Predictor(models, *Predictor.box_of(tr), tol=5e-4, envelope=Predictor.envelope_of(tr))
    P, fb, _ = pred(te.X, te.mom)
    e = np.max(np.abs(P - te.P), axis=1)
    sig = np.sqrt(te.P[:, 40] * (1 - te.P[:, 40]) / te.samples)
    res = {"train_examples": len(tr.X), "test_examples": len(te.X), "md_seconds": t1 - t0,
           "test_label_sigma_p0": {"median": float(np.median(sig)), "max": float(sig.max())},
           "train_seconds": t2 - t1, "loss": hist, "test": evaluate(models[0], te),
           "predictor": {"max": float(e.max()), "median": float(np.median(e)),
                         "q99": float(np.quantile(e, 0.99)), "fallback_fraction": float(fb.mean()),
                         "outside_envelope": float((~pred.trusted(te.X)).mean())},
           "inference": inference_throughput(models[0])}
    if save:
        np.savez_compressed(save, X=te.X, P=te.P, Wsg=te.Wsg, samples=te.samples, rep=te.rep, pred=P, fallback=fb)
    print(json.dumps(res))


if __name__ == "__main__":
    import sys

    main(sys.argv[sys.argv.index("--save") + 1] if "--save" in sys.argv else None)
