"""ctypes binding of the FP64 CPU oracle (oracle/mdlg_oracle.c, oracle/mlp_oracle.c).

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py.  Never imported by the product path.

``build()`` compiles the oracle with gcc (FP64, -ffp-contract=off so every
product and sum rounds on its own).  The wrappers take and return numpy arrays.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("mdlg_oracle.c", "mlp_oracle.c")]
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    srcs = [s for s in _SRCS if os.path.exists(s)]
    stale = force or not os.path.exists(_SO) or any(
        os.path.getmtime(s) > os.path.getmtime(_SO) for s in srcs)
    if stale:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, *srcs, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = C.CDLL(_SO)
            _declare(_lib)
    return _lib


P = C.c_void_p
I64 = C.c_int64
I32 = C.c_int32
D = C.c_double


def _declare(L):
    L.or_bin_xy.argtypes = [I64, P, P, P, P, D, I64, I32, P, P, P]
    L.or_bin_xy.restype = None
    L.or_bin_celloff.argtypes = [I64, P, P, P, P, P, P, I32, I32, D, D, I64, I32, P, P, P]
    L.or_bin_celloff.restype = C.c_int
    L.or_feq_g1.argtypes = [D, D]
    L.or_feq_g1.restype = D
    L.or_feq_gaussian.argtypes = [D, D, D, I32, P]
    L.or_feq_gaussian.restype = None
    L.or_wsg_cmax.argtypes = [D]
    L.or_wsg_cmax.restype = I32
    L.or_poisson.argtypes = [I32, D]
    L.or_poisson.restype = D
    L.or_feq_wsg1.argtypes = [D, D, D, I32]
    L.or_feq_wsg1.restype = D
    L.or_feq_wsg.argtypes = [D, D, D, D, I32, P]
    L.or_feq_wsg.restype = None
    L.or_wsg_mu4.argtypes = [D, D]
    L.or_wsg_mu4.restype = D
    L.or_wsg_lambda.argtypes = [D, D, P, P]
    L.or_wsg_lambda.restype = C.c_int
    L.or_kl.argtypes = [P, P, I64]
    L.or_kl.restype = D
    L.or_kl_terms.argtypes = [P, P, I64, P]
    L.or_kl_terms.restype = None
    L.or_site_occupation.argtypes = [I64, P, P, P, P, P, P, I32, I32, D, D, I64, I32, P, P]
    L.or_site_occupation.restype = C.c_int
    L.or_collision.argtypes = [P, P, I64, I32, P]
    L.or_collision.restype = None
    L.or_disp_hist.argtypes = [I64, P, P, P, P, P, P, I32, I32, D, D, D, I32, P, P]
    L.or_disp_hist.restype = C.c_int
    L.or_pdf_gauss_bins.argtypes = [D, D, I32, P]
    L.or_pdf_gauss_bins.restype = None
    L.or_pdf_wsg_bins.argtypes = [D, D, D, I32, P]
    L.or_pdf_wsg_bins.restype = None
    L.or_symmetrize.argtypes = [P, I32, P]
    L.or_symmetrize.restype = None
    L.or_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
    L.or_splitmix64.restype = C.c_uint64
    L.or_bootstrap_feq.argtypes = [P, P, I32, I32, D, I32, I32, C.c_uint64, I32, P]
    L.or_bootstrap_feq.restype = C.c_int
    L.or_lj_pair.argtypes = [D, D, D, D, P]
    L.or_lj_pair.restype = D
    L.or_forces_brute.argtypes = [I64, P, P, D, D, D, D, P, P, P, P]
    L.or_forces_brute.restype = None
    L.or_forces_cells.argtypes = [I64, P, P, D, D, D, D, P, P, P, P, I64, P]
    L.or_forces_cells.restype = C.c_int
    L.or_energy.argtypes = [I64, P, P, P, P, D, D, D, D, D, P]
    L.or_energy.restype = C.c_int
    L.or_md_run.argtypes = [I64, P, P, P, P, D, D, D, D, D, D, I64, I64,
                            I32, P, I32, P, I32, P, P, P, P, P]
    L.or_md_run.restype = C.c_int
    if hasattr(L, "or_mlp_forward"):
        _declare_mlp(L)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- binning
def bin_xy(x0, y0, x1, y1, L, lx, W):
    x0, y0, x1, y1 = map(_f64, (x0, y0, x1, y1))
    nb = (2 * W + 1) ** 2
    hist = np.zeros(nb, np.int64)
    ovf = np.zeros(1, np.int64)
    mom = np.zeros(2, np.float64)
    lib().or_bin_xy(len(x0), _p(x0), _p(y0), _p(x1), _p(y1), L, lx, W, _p(hist), _p(ovf), _p(mom))
    return hist, int(ovf[0]), mom


def bin_celloff(s, ncell, h, L, lx, W):
    """s: dict(cell0, ox0, oy0, cell1, ox1, oy1) as from inputs.random_celloff_snapshots."""
    f64 = s["ox0"].dtype == np.float64
    ft = np.float64 if f64 else np.float32
    arrs = [np.ascontiguousarray(s[k], dtype=(np.int32 if k.startswith("cell") else ft))
            for k in ("cell0", "ox0", "oy0", "cell1", "ox1", "oy1")]
    n = len(arrs[0])
    nb = (2 * W + 1) ** 2
    hist = np.zeros(nb, np.int64)
    ovf = np.zeros(1, np.int64)
    mom = np.zeros(2, np.float64)
    rc = lib().or_bin_celloff(n, *[_p(a) for a in arrs], int(f64), ncell, h, L, lx, W,
                              _p(hist), _p(ovf), _p(mom))
    assert rc == 0
    return hist, int(ovf[0]), mom


def site_occupation(s, ncell, h, L, lx, W):
    """Local occupation numbers of Eq. (n_i) for the snapshot pair s (t0 ->
    t1): returns (n int64[(2W+1)^2, lx, lx] indexed [class][ly][lx], ovf
    int64[lx, lx]) at the arrival sites."""
    f64 = s["ox0"].dtype == np.float64
    ft = np.float64 if f64 else np.float32
    arrs = [np.ascontiguousarray(s[k], dtype=(np.int32 if k.startswith("cell") else ft))
            for k in ("cell0", "ox0", "oy0", "cell1", "ox1", "oy1")]
    n = len(arrs[0])
    nb = (2 * W + 1) ** 2
    nf = np.zeros((nb, lx, lx), np.int64)
    ovf = np.zeros((lx, lx), np.int64)
    rc = lib().or_site_occupation(n, *[_p(a) for a in arrs], int(f64), ncell, h, L, lx, W,
                                  _p(nf), _p(ovf))
    assert rc == 0
    return nf, ovf


def collision(nt, nn, W):
    """Collision operator Xi of Eq. (mdlg_evolution) from the occupation
    fields at t and t + dt (layout of site_occupation)."""
    nt = np.ascontiguousarray(nt, dtype=np.int64)
    nn = np.ascontiguousarray(nn, dtype=np.int64)
    xi = np.zeros_like(nt)
    lib().or_collision(_p(nt), _p(nn), nt.shape[-1], W, _p(xi))
    return xi


def disp_hist(s, ncell, h, L, width, nbins):
    """Histogram of the continuous per-axis displacement (both axes) of the
    snapshot pair s over nbins bins of the given width centred on 0; returns
    (hist int64[nbins], outside)."""
    f64 = s["ox0"].dtype == np.float64
    ft = np.float64 if f64 else np.float32
    arrs = [np.ascontiguousarray(s[k], dtype=(np.int32 if k.startswith("cell") else ft))
            for k in ("cell0", "ox0", "oy0", "cell1", "ox1", "oy1")]
    hist = np.zeros(nbins, np.int64)
    out = np.zeros(1, np.int64)
    rc = lib().or_disp_hist(len(arrs[0]), *[_p(a) for a in arrs], int(f64), ncell, h, L, width,
                            nbins, _p(hist), _p(out))
    assert rc == 0
    return hist, int(out[0])


def pdf_gauss_bins(mu2, width, nbins):
    P_ = np.zeros(nbins)
    lib().or_pdf_gauss_bins(float(mu2), float(width), int(nbins), _p(P_))
    return P_


def pdf_wsg_bins(mu2, lam, width, nbins):
    P_ = np.zeros(nbins)
    lib().or_pdf_wsg_bins(float(mu2), float(lam), float(width), int(nbins), _p(P_))
    return P_


def kl_terms(R, Q):
    R, Q = _f64(R), _f64(Q)
    K = np.zeros(len(R))
    lib().or_kl_terms(_p(R), _p(Q), len(R), _p(K))
    return K


# ---------------------------------------------------------------- closed forms
def feq_g1(u, a2):
    return lib().or_feq_g1(float(u), float(a2))


def feq_gaussian(a2, ux=0.0, uy=0.0, W=4):
    P_ = np.zeros((2 * W + 1) ** 2)
    lib().or_feq_gaussian(a2, ux, uy, W, _p(P_))
    return P_


def feq_wsg1(u, a2, lam, c):
    return lib().or_feq_wsg1(float(u), float(a2), float(lam), int(c))


def feq_wsg(a2, lam, ux=0.0, uy=0.0, W=4):
    P_ = np.zeros((2 * W + 1) ** 2)
    lib().or_feq_wsg(a2, lam, ux, uy, W, _p(P_))
    return P_


def wsg_cmax(lam):
    return lib().or_wsg_cmax(float(lam))


def poisson(c, lam):
    return lib().or_poisson(int(c), float(lam))


def wsg_mu4(mu2, lam):
    return lib().or_wsg_mu4(mu2, lam)


def wsg_lambda(mu2, mu4):
    l1 = C.c_double()
    l2 = C.c_double()
    rc = lib().or_wsg_lambda(mu2, mu4, C.byref(l1), C.byref(l2))
    return rc, l1.value, l2.value


def kl(R, Q):
    R, Q = _f64(R), _f64(Q)
    return lib().or_kl(_p(R), _p(Q), len(R))


def symmetrize(P_, W):
    P_ = _f64(P_)
    out = np.zeros_like(P_)
    lib().or_symmetrize(_p(P_), W, _p(out))
    return out


def splitmix64(seed, c):
    return int(lib().or_splitmix64(seed & (2 ** 64 - 1), c & (2 ** 64 - 1)))


def bootstrap_feq(hist_blocks, wblk, W, n, sym=False, B=200, seed=0, rep=0):
    """Block-bootstrap standard error of the measured P_i (or_bootstrap_feq):
    hist_blocks int64 [nblk, (2W+1)^2], wblk int64 [nblk] windows per block."""
    h = np.ascontiguousarray(hist_blocks, dtype=np.int64)
    w = np.ascontiguousarray(wblk, dtype=np.int64)
    out = np.zeros((2 * W + 1) ** 2)
    rc = lib().or_bootstrap_feq(_p(h), _p(w), len(w), W, float(n), int(sym), int(B), seed & (2 ** 64 - 1), rep,
                                _p(out))
    assert rc == 0, rc
    return out


# ---------------------------------------------------------------- forces / MD
def lj_pair(r2, rc=2.5, eps=1.0, sigma=1.0):
    fr = C.c_double()
    v = lib().or_lj_pair(r2, rc, eps, sigma, C.byref(fr))
    return v, fr.value


def forces_brute(x, y, L, rc=2.5, eps=1.0, sigma=1.0):
    x, y = _f64(x), _f64(y)
    n = len(x)
    fx, fy, pe, fa = (np.zeros(n) for _ in range(4))
    lib().or_forces_brute(n, _p(x), _p(y), L, rc, eps, sigma, _p(fx), _p(fy), _p(pe), _p(fa))
    return fx, fy, pe, fa


def forces_cells(x, y, L, rc=2.5, eps=1.0, sigma=1.0, subset=None):
    x, y = _f64(x), _f64(y)
    n = len(x)
    fx, fy, pe, fa = (np.zeros(n) for _ in range(4))
    sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int64)
    rc_ = lib().or_forces_cells(n, _p(x), _p(y), L, rc, eps, sigma, _p(fx), _p(fy), _p(pe),
                                _p(fa), 0 if sub is None else len(sub), _p(sub))
    assert rc_ == 0, rc_
    return fx, fy, pe, fa


def energy(x, y, vx, vy, L, rc=2.5, eps=1.0, sigma=1.0, mass=1.0):
    x, y, vx, vy = map(_f64, (x, y, vx, vy))
    out = np.zeros(4)
    rc_ = lib().or_energy(len(x), _p(x), _p(y), _p(vx), _p(vy), L, rc, eps, sigma, mass, _p(out))
    assert rc_ == 0
    return out


def md_run(x, y, vx, vy, L, dt, nsteps, n_equil=0, every=(), lx=(), W=4, rc=2.5, eps=1.0,
           sigma=1.0, mass=1.0, energy_log=False):
    """Runs the oracle dynamics on copies of the state; returns a dict with the
    final state, histograms [n_lg][n_dx][nb], overflow [n_lg][n_dx],
    moments [n_lg][2], window counts [n_lg] and optionally the energy log."""
    x, y, vx, vy = (np.array(a, dtype=np.float64, copy=True) for a in (x, y, vx, vy))
    n = len(x)
    every = np.ascontiguousarray(every, dtype=np.int32)
    lxa = np.ascontiguousarray(lx, dtype=np.int64)
    nlg, ndx = len(every), len(lxa)
    nb = (2 * W + 1) ** 2
    hist = np.zeros((max(nlg, 1), max(ndx, 1), nb), np.int64)
    ovf = np.zeros((max(nlg, 1), max(ndx, 1)), np.int64)
    mom = np.zeros((max(nlg, 1), 2))
    nwin = np.zeros(max(nlg, 1), np.int64)
    elog = np.zeros((nsteps + 1, 4)) if energy_log else None
    rc_ = lib().or_md_run(n, _p(x), _p(y), _p(vx), _p(vy), L, rc, eps, sigma, mass, dt, nsteps,
                          n_equil, nlg, _p(every), ndx, _p(lxa), W, _p(hist), _p(ovf), _p(mom),
                          _p(nwin), _p(elog))
    assert rc_ == 0, rc_
    return dict(x=x, y=y, vx=vx, vy=vy, hist=hist[:nlg, :ndx], overflow=ovf[:nlg, :ndx],
                mom=mom[:nlg], nwin=nwin[:nlg], elog=elog)


# ---------------------------------------------------------------- MLP (surrogate)
def _declare_mlp(L):
    L.or_mlp_forward.argtypes = [I32, P, I64, P, P, P, P, P]
    L.or_mlp_forward.restype = C.c_int
    L.or_mlp_loss_backward.argtypes = [I32, P, I64, P, P, P, P, P, P]
    L.or_mlp_loss_backward.restype = D


def mlp_pack(Ws, bs):
    """Packs [W_1, b_1, W_2, b_2, ...] (W row-major [out][in]) into one FP64 vector."""
    return np.concatenate([np.concatenate([np.asarray(W, np.float64).ravel(),
                                           np.asarray(b, np.float64).ravel()])
                           for W, b in zip(Ws, bs)])


def mlp_forward(sizes, X, params, shift, scale):
    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    X = _f64(X)
    M = X.shape[0]
    out = np.zeros((M, int(sizes[-1])))
    rc = lib().or_mlp_forward(len(sizes) - 1, _p(sizes), M, _p(X), _p(_f64(shift)), _p(_f64(scale)),
                              _p(_f64(params)), _p(out))
    assert rc == 0
    return out


def mlp_loss_backward(sizes, X, params, T, shift, scale):
    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    X = _f64(X)
    params = _f64(params)
    grad = np.zeros_like(params)
    loss = lib().or_mlp_loss_backward(len(sizes) - 1, _p(sizes), X.shape[0], _p(X),
                                      _p(_f64(shift)), _p(_f64(scale)), _p(params), _p(_f64(T)),
                                      _p(grad))
    return loss, grad
