"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds input generation only (initial states, random snapshots,
ensemble parameter draws, surrogate query points).  It contains none of the
method's arithmetic: no forces, no integration, no lattice mapping, no
equilibrium formulas.  Every generator takes an explicit integer seed and uses
numpy's PCG64, so the same call yields bit-identical arrays on every machine.

The initial state follows the paper's set-up (Sec. 4): homogeneously placed
particles with kinetic energy matching the temperature and zero total
momentum; the placement recipe (square lattice with uniform jitter, Maxwell
velocities, exact kinetic-energy rescale) is the synthetic stand-in stated in
the design notes.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def box_length(n: int, phi: float, sigma: float = 1.0) -> float:
    """Edge of the periodic square box holding ``n`` disks of diameter sigma
    at area fraction ``phi`` (area fraction definition of Sec. 4)."""
    return math.sqrt(n * math.pi * sigma * sigma / (4.0 * phi))


@dataclass
class State:
    x: np.ndarray
    y: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    L: float


def lattice_gas_state(n: int, L: float, T: float, seed: int, jitter: float = 0.1,
                      mass: float = 1.0) -> State:
    """Square lattice of ceil(sqrt(n))^2 sites (row-major, first n used),
    spacing L/ceil(sqrt(n)), each site shifted by a uniform jitter in
    [-jitter, jitter) per axis; Maxwell velocities at temperature T with the
    mean removed and the kinetic energy rescaled to exactly (2n-2) T / 2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = int(math.ceil(math.sqrt(n)))
    a = L / m
    idx = np.arange(n, dtype=np.int64)
    ix = idx % m
    iy = idx // m
    x = (ix + 0.5) * a + rng.uniform(-jitter, jitter, n)
    y = (iy + 0.5) * a + rng.uniform(-jitter, jitter, n)
    x = np.mod(x, L)
    y = np.mod(y, L)
    x[x >= L] -= L
    y[y >= L] -= L
    vx, vy = _maxwell(rng, n, T, mass)
    return State(x, y, vx, vy, L)


def _maxwell(rng, n, T, mass):
    s = math.sqrt(T / mass)
    vx = rng.normal(0.0, s, n)
    vy = rng.normal(0.0, s, n)
    if n > 1:
        vx -= vx.mean()
        vy -= vy.mean()
        ke = 0.5 * mass * float(np.sum(vx * vx) + np.sum(vy * vy))
        target = (2 * n - 2) * T / 2.0
        if ke > 0:
            f = math.sqrt(target / ke)
            vx *= f
            vy *= f
    return vx, vy


def ideal_gas_state(n: int, L: float, T: float, seed: int, mass: float = 1.0) -> State:
    """Uniformly random positions and Maxwell velocities (no rescale): the
    input of the non-interacting (ballistic) special case."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(0.0, L, n)
    y = rng.uniform(0.0, L, n)
    s = math.sqrt(T / mass)
    vx = rng.normal(0.0, s, n)
    vy = rng.normal(0.0, s, n)
    return State(x, y, vx, vy, L)


def random_celloff_snapshots(n: int, ncell: int, h: float, seed: int, max_step: float,
                             f64: bool = False, ties: int = 0, lattice_dx: float | None = None):
    """A pair of snapshots in the (linear cell index, in-cell offset) encoding.

    Snapshot 0 is uniform over the box; snapshot 1 moves each particle by a
    random displacement of at most ``max_step`` per axis, re-expressed in the
    cell it lands in, with offsets deliberately allowed up to 0.25 h outside
    [0, h) as a stale cell list produces.  ``ties`` particles of snapshot 0 are
    placed exactly on lattice-line multiples of ``lattice_dx`` (boundary ties).
    Returns dict(cell0, ox0, oy0, cell1, ox1, oy1) as numpy arrays.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ft = np.float64 if f64 else np.float32
    cx0 = rng.integers(0, ncell, n)
    cy0 = rng.integers(0, ncell, n)
    ox0 = rng.uniform(0.0, h, n).astype(ft)
    oy0 = rng.uniform(0.0, h, n).astype(ft)
    if ties and lattice_dx is not None:
        k = min(ties, n)
        L = ncell * h
        nl = int(L // lattice_dx)
        for i in range(k):
            j = int(rng.integers(0, max(nl, 1)))
            xt = j * lattice_dx
            c = int(xt // h)
            c = min(max(c, 0), ncell - 1)
            cx0[i] = c
            ox0[i] = ft(xt - c * h)
    dx = rng.uniform(-max_step, max_step, n)
    dy = rng.uniform(-max_step, max_step, n)
    # land cell: shift by whole cells, keep a jittered non-canonical offset
    X = cx0 * h + ox0.astype(np.float64) + dx
    Y = cy0 * h + oy0.astype(np.float64) + dy
    slack_x = rng.uniform(-0.25, 0.25, n) * h
    slack_y = rng.uniform(-0.25, 0.25, n) * h
    cx1 = np.floor((X - slack_x) / h).astype(np.int64)
    cy1 = np.floor((Y - slack_y) / h).astype(np.int64)
    ox1 = (X - cx1 * h).astype(ft)
    oy1 = (Y - cy1 * h).astype(ft)
    cx1 %= ncell
    cy1 %= ncell
    return dict(
        cell0=(cy0 * ncell + cx0).astype(np.int32), ox0=ox0, oy0=oy0,
        cell1=(cy1 * ncell + cx1).astype(np.int32), ox1=ox1, oy1=oy1,
    )


def random_celloff_walk(n: int, ncell: int, h: float, seed: int, max_step: float, steps: int,
                        f64: bool = False):
    """``steps`` + 1 snapshots of a random walk in the (linear cell index,
    in-cell offset) encoding: uniform start, then per snapshot a uniform
    displacement of at most ``max_step`` per axis, re-expressed in the cell it
    lands in with offsets up to 0.25 h outside [0, h) (a stale cell list).
    Returns a list of dict(cell, ox, oy)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ft = np.float64 if f64 else np.float32
    L = ncell * h
    X = rng.uniform(0.0, L, n)
    Y = rng.uniform(0.0, L, n)
    out = []
    for k in range(steps + 1):
        if k:
            X = np.mod(X + rng.uniform(-max_step, max_step, n), L)
            Y = np.mod(Y + rng.uniform(-max_step, max_step, n), L)
        sx = rng.uniform(-0.25, 0.25, n) * h
        sy = rng.uniform(-0.25, 0.25, n) * h
        cx = np.floor((X - sx) / h).astype(np.int64)
        cy = np.floor((Y - sy) / h).astype(np.int64)
        ox = (X - cx * h).astype(ft)
        oy = (Y - cy * h).astype(ft)
        out.append(dict(cell=((cy % ncell) * ncell + (cx % ncell)).astype(np.int32), ox=ox, oy=oy))
    return out


def shear_wave_state(n: int, L: float, T: float, U: float, seed: int) -> State:
    """lattice_gas_state with a transverse sine flow added: vx += U sin(2 pi
    y / L) (one wavelength over the box), less its mean so that the total
    momentum stays zero."""
    st = lattice_gas_state(n, L, T, seed)
    w = U * np.sin(2.0 * np.pi * st.y / L)
    st.vx = st.vx + (w - w.mean())
    return st


def ensemble_params(n_rep: int, seed: int, n_min: int = 4096, n_max: int = 65536,
                    phi_lo: float = 0.02, phi_hi: float = 0.30, T_lo: float = 1.0,
                    T_hi: float = 20.0):
    """Replica draws of the batched ensemble: N log-uniform in [n_min, n_max],
    area fraction uniform in [phi_lo, phi_hi], T uniform in [T_lo, T_hi].
    Returns (N int64[n_rep], phi float64[n_rep], T float64[n_rep])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(0.0, 1.0, n_rep)
    N = np.floor(n_min * (n_max / n_min) ** u).astype(np.int64)
    N = np.clip(N, n_min, n_max)
    phi = rng.uniform(phi_lo, phi_hi, n_rep)
    T = rng.uniform(T_lo, T_hi, n_rep)
    return N, phi, T


def surrogate_queries(n: int, seed: int, lo=(0.02, 1.0, 0.05, 0.5), hi=(0.30, 20.0, 1.0, 2.0)):
    """Uniform query points (phi, T, dt_lg, dx) in the training box, float32 [n, 4]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    q = lo + (hi - lo) * rng.uniform(0.0, 1.0, (n, 4))
    return q.astype(np.float32)


def mlp_init(layer_sizes, seed: int):
    """He-uniform initial weights (float32, row-major [out, in]) and zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ws, bs = [], []
    for fan_in, fan_out in zip(layer_sizes[:-1], layer_sizes[1:]):
        lim = math.sqrt(6.0 / fan_in)
        Ws.append(rng.uniform(-lim, lim, (fan_out, fan_in)).astype(np.float32))
        bs.append(np.zeros(fan_out, dtype=np.float32))
    return Ws, bs
