"""Thin Python binding of libmdlg.so (C-ABI in include/mdlg.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (their data_ptr() is passed);
streams are torch streams (the current stream by default).  If the library is
missing this module raises instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libmdlg.so")
_lib = None

MD_OK = 0
MD_E_ARG, MD_E_CUDA, MD_E_TIMEOUT, MD_E_SKIN, MD_E_NONFINITE, MD_E_DOMAIN, MD_E_NOMEM, MD_E_LIMIT = \
    -1, -2, -3, -4, -5, -6, -7, -8
MD_FP64, MD_FP32_CELLOFF = 0, 1
MD_MAX_LG, MD_MAX_DX, MD_MAX_W, MD_NBLK, MD_MAX_REP = 8, 4, 10, 32, 4096


class MDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libmdlg error {code}: {msg}")
        self.code = code


class md_params(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("box_L", C.c_double), ("dt", C.c_double), ("rc", C.c_double),
        ("eps", C.c_double), ("sigma", C.c_double), ("mass", C.c_double), ("skin", C.c_double),
        ("precision", C.c_int32), ("W", C.c_int32), ("n_equil", C.c_int64),
        ("n_lg", C.c_int32), ("lg_every", C.c_int32 * MD_MAX_LG),
        ("n_dx", C.c_int32), ("lx", C.c_int32 * MD_MAX_DX),
        ("block_windows", C.c_int32), ("nbr_max", C.c_int32),
    ]


class md_snapshot(C.Structure):
    _fields_ = [("cell", C.c_void_p), ("off_x", C.c_void_p), ("off_y", C.c_void_p),
                ("off_is_f64", C.c_int32), ("ncell", C.c_int32), ("h", C.c_double)]


class md_info_t(C.Structure):
    _fields_ = [("n_total", C.c_int64), ("step", C.c_int64), ("n_rebuilds", C.c_int64),
                ("n_rep", C.c_int32), ("precision", C.c_int32), ("grid_blocks", C.c_int32),
                ("block_threads", C.c_int32)]


class md_rep_info_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("L_eff", C.c_double), ("h", C.c_double),
                ("ncell", C.c_int32), ("reserved", C.c_int32),
                ("dx_eff", C.c_double * MD_MAX_DX)]


class md_feq_stats(C.Structure):
    _fields_ = [("mu2", C.c_double), ("mu4", C.c_double), ("a2", C.c_double),
                ("dx_eff", C.c_double), ("n_windows", C.c_int64), ("n_samples", C.c_int64),
                ("n_overflow", C.c_int64), ("n_blocks_used", C.c_int64)]


P = C.c_void_p
_SIGS = {
    "md_init": ([C.POINTER(md_params), P, P, P, P, P, C.POINTER(P)], C.c_int),
    "md_init_batch": ([C.POINTER(md_params), C.c_int32, P, P, P, P, P, C.POINTER(P)], C.c_int),
    "md_destroy": ([P], None),
    "md_step": ([P, C.c_int64], C.c_int),
    "md_sync": ([P], C.c_int),
    "md_barrier_selftest": ([P, C.c_double], C.c_int),
    "md_resident_plan": ([C.POINTER(md_params), C.c_int32, C.c_int32, C.c_int64, P, C.c_int32, P, P], C.c_int),
    "md_tune": ([P, C.c_int32, C.c_int32, C.c_int32], C.c_int),
    "md_autotune": ([P, C.c_int64, P], C.c_int),
    "md_info": ([P, C.POINTER(md_info_t)], C.c_int),
    "md_rep_info": ([P, C.c_int32, C.POINTER(md_rep_info_t)], C.c_int),
    "md_get_state": ([P, P, P, P, P], C.c_int),
    "md_set_state": ([P, P, P, P, P], C.c_int),
    "md_get_raw": ([P, P, P, P], C.c_int),
    "md_get_snapshot": ([P, C.c_int32, P, P, P], C.c_int),
    "md_forces": ([P, P, P, P], C.c_int),
    "md_step_forces": ([P, C.c_int64, P, P], C.c_int),
    "md_energy": ([P, C.c_int32, P], C.c_int),
    "md_energy_batch": ([P, P], C.c_int),
    "md_checkpoint_bytes": ([P, C.POINTER(C.c_int64)], C.c_int),
    "md_checkpoint_save": ([P, P], C.c_int),
    "md_checkpoint_load": ([P, P], C.c_int),
    "md_hist_raw": ([P, C.c_int32, C.c_int32, C.c_int32, P, P, P], C.c_int),
    "feq_measured": ([P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, P,
                      C.POINTER(md_feq_stats)], C.c_int),
    "feq_batch": ([P, C.c_int32, C.c_int32, C.c_int32, P], C.c_int),
    "md_hist_blocks": ([P, C.c_int32, C.c_int32, C.c_int32, P, P], C.c_int),
    "feq_bootstrap": ([P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, P], C.c_int),
    "mdlg_bin": ([C.POINTER(md_snapshot), C.POINTER(md_snapshot), C.c_int64, C.c_int32, C.c_int32,
                  P, P, P, P], C.c_int),
    "mdlg_bin_noalloc": ([C.POINTER(md_snapshot), C.POINTER(md_snapshot), C.c_int64, C.c_int32,
                          C.c_int32, P, P, P, P], C.c_int),
    "mdlg_disp_hist": ([C.POINTER(md_snapshot), C.POINTER(md_snapshot), C.c_int64, C.c_double,
                        C.c_int32, P, P, P], C.c_int),
    "mdlg_site_occupation": ([C.POINTER(md_snapshot), C.POINTER(md_snapshot), C.c_int64, C.c_int32,
                              C.c_int32, P, P, P], C.c_int),
    "mdlg_collision": ([P, P, C.c_int32, C.c_int32, C.c_double, P, P, P], C.c_int),
    "disp_pdf_models": ([C.c_double, C.c_double, C.c_double, C.c_int32, P, P, P], C.c_int),
    "kl_terms": ([P, P, C.c_int32, P, P], C.c_int),
    "feq_gaussian": ([C.c_double, C.c_double, C.c_double, C.c_int32, P, P], C.c_int),
    "wsg_lambda": ([C.c_double, C.c_double, C.c_int32, P, P], C.c_int),
    "feq_wsg": ([C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32, P, P], C.c_int),
    "feq_compare": ([P, P, C.c_int32, P, P], C.c_int),
    "md_last_error": ([], C.c_char_p),
    "mdlg_fma_peak": ([C.c_int32, C.c_int64, P, P, P], C.c_int),
    "mlp_create": ([C.c_int32, C.c_int32, C.c_int32, P, P, P, C.POINTER(P)], C.c_int),
    "mlp_destroy": ([P], None),
    "mlp_param_count": ([P], C.c_int64),
    "mlp_set_params": ([P, P], C.c_int),
    "mlp_get_params": ([P, P], C.c_int),
    "mlp_forward": ([P, P, C.c_int64, P, P], C.c_int),
    "mlp_grad": ([P, P, P, C.c_int32, P, P, P], C.c_int),
    "mlp_train_step": ([P, P, P, C.c_int32, C.c_float, P, P], C.c_int),
    "mlp_status": ([P], C.c_int),
    "bf16_gemm_tn": ([P, P, P, C.c_int32, C.c_int32, C.c_int32, P, P], C.c_int),
    "bf16_gemm_selftest": ([P, P, P, C.c_int32, C.c_int32, C.c_int32, P, C.c_double, P], C.c_int),
}


def library_path() -> str:
    return _SO


def load():
    """Loads libmdlg.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise ImportError(f"libmdlg.so not built ({_SO}); run __graft_entry__.build()")
        lib = C.CDLL(_SO)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _check(rc):
    if rc != MD_OK:
        msg = load().md_last_error().decode(errors="replace")
        raise MDError(rc, msg)
    return rc


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(a):
    """Device pointer of a torch tensor, or host pointer of a numpy array."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return C.c_void_p(a.ctypes.data)
    assert a.is_contiguous()
    return C.c_void_p(a.data_ptr())


def make_params(n, L, dt=5e-4, rc=2.5, eps=1.0, sigma=1.0, mass=1.0, skin=0.5,
                precision=MD_FP32_CELLOFF, W=4, n_equil=0, lg_every=(400,), lx=(101,),
                block_windows=1) -> md_params:
    p = md_params()
    p.n, p.box_L, p.dt, p.rc, p.eps, p.sigma, p.mass, p.skin = n, L, dt, rc, eps, sigma, mass, skin
    p.precision, p.W, p.n_equil = precision, W, n_equil
    p.n_lg = len(lg_every)
    for k, v in enumerate(lg_every):
        p.lg_every[k] = int(v)
    p.n_dx = len(lx)
    for k, v in enumerate(lx):
        p.lx[k] = int(v)
    p.block_windows = block_windows
    return p


class System:
    """A system of one or more replicas (md_init / md_init_batch)."""

    def __init__(self, params, x, y, vx, vy, stream=None):
        lib = load()
        if isinstance(params, md_params):
            params = [params]
        self.params = list(params)
        arr = (md_params * len(self.params))(*self.params)
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) if isinstance(a, np.ndarray) else a
                      for a in (x, y, vx, vy)]
        h = P()
        self._stream = _stream(stream)
        _check(lib.md_init_batch(arr, len(self.params), *[_ptr(a) for a in self._keep],
                                 self._stream, C.byref(h)))
        self.h = h
        self._keep = None
        self.n_total = int(sum(p.n for p in self.params))
        self.prec = self.params[0].precision
        self.nb = (2 * self.params[0].W + 1) ** 2

    def close(self):
        if getattr(self, "h", None):
            load().md_destroy(self.h)
            self.h = None

    __del__ = close

    def step(self, nsteps):
        _check(load().md_step(self.h, int(nsteps)))

    def sync(self):
        _check(load().md_sync(self.h))

    def barrier_selftest(self, limit_s=0.02):
        """Return code of md_barrier_selftest (MD_E_TIMEOUT when the bounded
        barrier wait works); the system must be closed afterwards."""
        return int(load().md_barrier_selftest(self.h, float(limit_s)))

    def tune(self, block_threads=0, per_thread=0, staging=0):
        _check(load().md_tune(self.h, block_threads, per_thread, staging))

    def autotune(self, steps_per_trial=100):
        best = np.zeros(3, np.int32)
        _check(load().md_autotune(self.h, int(steps_per_trial), _ptr(best)))
        return tuple(int(v) for v in best)

    def info(self):
        o = md_info_t()
        _check(load().md_info(self.h, C.byref(o)))
        return o

    def rep_info(self, rep=0):
        o = md_rep_info_t()
        _check(load().md_rep_info(self.h, rep, C.byref(o)))
        return o

    def get_state(self):
        out = [np.zeros(self.n_total) for _ in range(4)]
        _check(load().md_get_state(self.h, *[_ptr(a) for a in out]))
        return out

    def set_state(self, x, y, vx, vy):
        """Host arrays (converted to FP64), or contiguous FP64 CUDA tensors
        of n_total elements each, read on the system's stream (the caller
        orders any copy into them before the call)."""
        arrs = (x, y, vx, vy)
        if all(getattr(a, "is_cuda", False) for a in arrs):
            import torch

            for a in arrs:
                if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != self.n_total:
                    raise ValueError(f"set_state: device arrays must be contiguous float64 of {self.n_total}")
        else:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
            if any(a.size != self.n_total for a in arrs):
                raise ValueError(f"set_state: arrays must hold {self.n_total} values")
        _check(load().md_set_state(self.h, *[_ptr(a) for a in arrs]))

    def _raw_buffers(self):
        import torch

        ft = torch.float64 if self.prec == MD_FP64 else torch.float32
        cell = torch.empty(self.n_total, dtype=torch.int32, device="cuda")
        ox = torch.empty(self.n_total, dtype=ft, device="cuda")
        oy = torch.empty(self.n_total, dtype=ft, device="cuda")
        return cell, ox, oy

    def get_raw(self):
        cell, ox, oy = self._raw_buffers()
        _check(load().md_get_raw(self.h, _ptr(cell), _ptr(ox), _ptr(oy)))
        return cell, ox, oy

    def get_snapshot(self, lg):
        cell, ox, oy = self._raw_buffers()
        _check(load().md_get_snapshot(self.h, lg, _ptr(cell), _ptr(ox), _ptr(oy)))
        return cell, ox, oy

    def forces(self):
        fx, fy, fa = (np.zeros(self.n_total) for _ in range(3))
        _check(load().md_forces(self.h, _ptr(fx), _ptr(fy), _ptr(fa)))
        return fx, fy, fa

    def step_forces(self, nsteps=1):
        """Advances nsteps and returns the list forces of the last step's
        force pass, FP64 by particle id (md_step_forces)."""
        fx, fy = np.zeros(self.n_total), np.zeros(self.n_total)
        _check(load().md_step_forces(self.h, int(nsteps), _ptr(fx), _ptr(fy)))
        return fx, fy

    def checkpoint(self):
        """Exact checkpoint (md_checkpoint_save) as a host byte array."""
        n = C.c_int64()
        _check(load().md_checkpoint_bytes(self.h, C.byref(n)))
        buf = np.empty(n.value, np.uint8)
        _check(load().md_checkpoint_save(self.h, _ptr(buf)))
        return buf

    def restore(self, buf):
        """Restores a checkpoint of a system with the same parameters."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(load().md_checkpoint_load(self.h, _ptr(buf)))

    def energy(self, rep=0):
        out = np.zeros(4)
        _check(load().md_energy(self.h, rep, _ptr(out)))
        return out

    def energy_batch(self):
        """[n_rep, 4] (kinetic, shifted potential, P_x, P_y) of every replica,
        from one evaluation of the state; row r equals energy(r) bit for bit."""
        out = np.zeros((len(self.params), 4))
        _check(load().md_energy_batch(self.h, _ptr(out)))
        return out

    def hist_raw(self, rep=0, lg=0, dxi=0):
        hist = np.zeros(self.nb, np.int64)
        ov = C.c_int64()
        nw = C.c_int64()
        _check(load().md_hist_raw(self.h, rep, lg, dxi, _ptr(hist), C.byref(ov), C.byref(nw)))
        return hist, ov.value, nw.value

    def feq_measured(self, rep=0, lg=0, dxi=0, symmetrize=False):
        Pm = np.zeros(self.nb)
        se = np.zeros(self.nb)
        st = md_feq_stats()
        _check(load().feq_measured(self.h, rep, lg, dxi, int(symmetrize), _ptr(Pm), _ptr(se),
                                   C.byref(st)))
        return Pm, se, st


def resident_plan(params, grid, smem_bytes, max_jobs=1 << 16):
    """Host-only dry run of the resident engine's plan (md_resident_plan):
    (jobs int32 [n, 8] = replica, g, k, r0, r1, p_cap, h_cap, cta0; grouped by
    CTA in execution order, start int32 [grid + 1], makespan)."""
    params = list(params)
    arr = (md_params * len(params))(*params)
    jobs = np.zeros((max_jobs, 8), np.int32)
    start = np.zeros(grid + 1, np.int32)
    ms = C.c_double()
    _check(load().md_resident_plan(arr, len(params), int(grid), int(smem_bytes), _ptr(jobs), max_jobs,
                                   _ptr(start), C.byref(ms)))
    return jobs[:start[-1]].copy(), start, ms.value


FEQB_STATS = 16
FEQB_FIELDS = ("mu2", "mu4", "a2", "lambda", "maxabs_g", "kl_g", "maxabs_wsg", "kl_wsg",
               "n_windows", "n_samples", "n_overflow", "dx_eff", "lambda_status", "sum_p")


def feq_batch(system, lg=0, dxi=0, symmetrize=True, out=None):
    """Batched f_eq stage; returns (P_md, P_g, P_wsg, stats) as arrays of shape
    [n_rep, nb] / [n_rep, 16] (host), or fills a device tensor `out`."""
    nrep = len(system.params)
    nb = system.nb
    stride = 3 * nb + FEQB_STATS
    if out is not None:
        _check(load().feq_batch(system.h, lg, dxi, int(symmetrize), _ptr(out)))
        return out
    buf = np.zeros((nrep, stride))
    _check(load().feq_batch(system.h, lg, dxi, int(symmetrize), _ptr(buf)))
    return buf[:, :nb], buf[:, nb:2 * nb], buf[:, 2 * nb:3 * nb], buf[:, 3 * nb:]


def hist_blocks(system, rep=0, lg=0, dxi=0):
    """Integer histogram per error-bar block: (int32 [MD_NBLK, nb], int64
    windows per block [MD_NBLK])."""
    h = np.zeros((MD_NBLK, system.nb), np.int32)
    w = np.zeros(MD_NBLK, np.int64)
    _check(load().md_hist_blocks(system.h, rep, lg, dxi, _ptr(h), _ptr(w)))
    return h, w


def feq_bootstrap(system, lg=0, dxi=0, symmetrize=False, n_resamples=200, seed=0):
    """Block-bootstrap standard error of P_i for every replica: [n_rep, nb]."""
    out = np.zeros((len(system.params), system.nb))
    _check(load().feq_bootstrap(system.h, lg, dxi, int(symmetrize), int(n_resamples),
                                C.c_uint64(seed & (2 ** 64 - 1)), _ptr(out)))
    return out


def _snapshots(cell0, ox0, oy0, cell1, ox1, oy1, ncell, h):
    """Checks a snapshot pair (the C ABI sees only pointers and one length)
    and returns (md_snapshot t0, md_snapshot t1, n): int32 cells and FP32 or
    FP64 offsets of one dtype, all 1-D, contiguous, of equal length, on the
    GPU.  Raises ValueError before any library call."""
    import torch

    arrs = (cell0, ox0, oy0, cell1, ox1, oy1)
    if not all(isinstance(a, torch.Tensor) for a in arrs):
        raise ValueError("snapshot arrays must be torch tensors")
    n = cell0.numel()
    if any(a.dim() != 1 or a.numel() != n or not a.is_contiguous() for a in arrs):
        raise ValueError("snapshot arrays must be contiguous 1-D tensors of one length")
    if cell0.dtype != torch.int32 or cell1.dtype != torch.int32:
        raise ValueError("snapshot cells must be int32")
    if ox0.dtype not in (torch.float32, torch.float64) or any(a.dtype != ox0.dtype for a in (oy0, ox1, oy1)):
        raise ValueError("snapshot offsets must all be float32 or all float64")
    if any(a.device.type != "cuda" for a in arrs) or len({a.device for a in arrs}) != 1:
        raise ValueError("snapshot arrays must be on one CUDA device")
    f64 = int(ox0.dtype == torch.float64)
    s0 = md_snapshot(_ptr(cell0).value, _ptr(ox0).value, _ptr(oy0).value, f64, int(ncell), float(h))
    s1 = md_snapshot(_ptr(cell1).value, _ptr(ox1).value, _ptr(oy1).value, f64, int(ncell), float(h))
    return s0, s1, n


def _field(t, shape, name, device):
    import torch

    if not isinstance(t, torch.Tensor) or t.dtype != torch.int32 or tuple(t.shape) != tuple(shape) \
            or not t.is_contiguous() or t.device != device:
        raise ValueError(f"{name} must be a contiguous int32 tensor of shape {tuple(shape)} on {device}")
    return t


def mdlg_bin(cell0, ox0, oy0, cell1, ox1, oy1, ncell, h, lx, W, stream=None, noalloc=False):
    """Histogram of lattice displacements between two device snapshots.
    noalloc=True calls mdlg_bin_noalloc (library-owned scratch; the outputs
    are still allocated here by torch)."""
    import torch

    s0, s1, n = _snapshots(cell0, ox0, oy0, cell1, ox1, oy1, ncell, h)
    dev = cell0.device
    nb = (2 * W + 1) ** 2
    hist = torch.empty(nb, dtype=torch.int32, device=dev)
    ovf = torch.empty(1, dtype=torch.int64, device=dev)
    mom = torch.empty(2, dtype=torch.float64, device=dev)
    fn = load().mdlg_bin_noalloc if noalloc else load().mdlg_bin
    _check(fn(C.byref(s0), C.byref(s1), n, lx, W, _ptr(hist), _ptr(ovf), _ptr(mom), _stream(stream)))
    return hist, ovf, mom


def disp_hist(cell0, ox0, oy0, cell1, ox1, oy1, ncell, h, width, nbins, stream=None):
    """Histogram of the continuous per-axis displacement between two device
    snapshots (Sec. 3(b), Fig. 2): (int64 tensor [nbins], outside count tensor)."""
    import torch

    s0, s1, n = _snapshots(cell0, ox0, oy0, cell1, ox1, oy1, ncell, h)
    hist = torch.empty(int(nbins), dtype=torch.int64, device=cell0.device)
    out = torch.empty(1, dtype=torch.int64, device=cell0.device)
    _check(load().mdlg_disp_hist(C.byref(s0), C.byref(s1), n, float(width), int(nbins),
                                 _ptr(hist), _ptr(out), _stream(stream)))
    return hist, out


def site_occupation(cell0, ox0, oy0, cell1, ox1, oy1, ncell, h, lx, W, field=None, ovf=None,
                    stream=None):
    """Local occupation numbers n_i(x, t1) of Eq. n_i between two device
    snapshots: (int32 field [(2W+1)^2, lx, lx], int32 overflow [lx, lx]).
    Given `field` / `ovf` tensors are added to (ensemble or window sums);
    otherwise zeroed ones are made."""
    import torch

    lx, W = int(lx), int(W)
    if lx < 1 or not 0 <= W <= MD_MAX_W:
        raise ValueError("site_occupation: lx >= 1 and 0 <= W <= MD_MAX_W")
    q = (2 * W + 1) ** 2
    if q * lx * lx >= 1 << 31:
        raise ValueError("site_occupation: (2W+1)^2 lx^2 must be < 2^31")
    s0, s1, n = _snapshots(cell0, ox0, oy0, cell1, ox1, oy1, ncell, h)
    dev = cell0.device
    field = torch.zeros((q, lx, lx), dtype=torch.int32, device=dev) if field is None else \
        _field(field, (q, lx, lx), "field", dev)
    ovf = torch.zeros((lx, lx), dtype=torch.int32, device=dev) if ovf is None else \
        _field(ovf, (lx, lx), "ovf", dev)
    _check(load().mdlg_site_occupation(C.byref(s0), C.byref(s1), n, lx, W, _ptr(field), _ptr(ovf),
                                       _stream(stream)))
    return field, ovf


def collision(n_t, n_next, W, scale=None, stream=None):
    """Collision operator of Eq. mdlg_evolution from two occupation fields:
    the int32 Xi field, or, with `scale` given, the float64 scale * Xi (the
    ensemble-averaged Omega for fields summed over 1/scale replicas)."""
    import torch

    W = int(W)
    if not 0 <= W <= MD_MAX_W:
        raise ValueError("collision: 0 <= W <= MD_MAX_W")
    if not isinstance(n_t, torch.Tensor) or n_t.dim() != 3:
        raise ValueError("collision: n_t must be a [(2W+1)^2, lx, lx] int32 tensor")
    lx = n_t.shape[-1]
    shape = ((2 * W + 1) ** 2, lx, lx)
    _field(n_t, shape, "n_t", n_t.device)
    _field(n_next, shape, "n_next", n_t.device)
    if n_t.device.type != "cuda":
        raise ValueError("collision: fields must be on a CUDA device")
    if scale is None:
        out = torch.empty_like(n_t)
        _check(load().mdlg_collision(_ptr(n_t), _ptr(n_next), int(lx), int(W), 1.0, _ptr(out), None,
                                     _stream(stream)))
    else:
        out = torch.empty(n_t.shape, dtype=torch.float64, device=n_t.device)
        _check(load().mdlg_collision(_ptr(n_t), _ptr(n_next), int(lx), int(W), float(scale), None,
                                     _ptr(out), _stream(stream)))
    return out


def disp_pdf_models(mu2, lam, width, nbins, stream=None):
    """Gaussian and Poisson-WSG bin masses over the bins of disp_hist."""
    import torch

    pg = torch.empty(nbins, dtype=torch.float64, device="cuda")
    pw = torch.empty(nbins, dtype=torch.float64, device="cuda")
    _check(load().disp_pdf_models(float(mu2), float(lam), float(width), int(nbins), _ptr(pg), _ptr(pw),
                                  _stream(stream)))
    return pg, pw


def kl_terms(R, Q, stream=None):
    """K(X_i) of Eq. k_Xi for device float64 tensors R, Q."""
    import torch

    K = torch.empty_like(R)
    _check(load().kl_terms(_ptr(R), _ptr(Q), R.numel(), _ptr(K), _stream(stream)))
    return K


def feq_gaussian(a2, ux=0.0, uy=0.0, W=4, stream=None):
    import torch

    out = torch.empty((2 * W + 1) ** 2, dtype=torch.float64, device="cuda")
    _check(load().feq_gaussian(a2, ux, uy, W, _ptr(out), _stream(stream)))
    return out


def wsg_lambda(mu2, mu4, root=2, stream=None, allow_domain=False):
    import torch

    out = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = load().wsg_lambda(mu2, mu4, root, _ptr(out), _stream(stream))
    if not (allow_domain and rc == MD_E_DOMAIN):
        _check(rc)
    return out, rc


def feq_wsg(a2, lam, ux=0.0, uy=0.0, W=4, stream=None):
    import torch

    out = torch.empty((2 * W + 1) ** 2, dtype=torch.float64, device="cuda")
    _check(load().feq_wsg(a2, lam, ux, uy, W, _ptr(out), _stream(stream)))
    return out


def feq_compare(R, Q, stream=None):
    import torch

    out = torch.empty(3, dtype=torch.float64, device="cuda")
    _check(load().feq_compare(_ptr(R), _ptr(Q), R.numel(), _ptr(out), _stream(stream)))
    return out


def fma_peak(f64, iters=1 << 16, stream=None):
    """Measured FMA throughput (flop/s) and the timed launch's ms."""
    f = C.c_double()
    ms = C.c_double()
    _check(load().mdlg_fma_peak(int(f64), int(iters), C.byref(f), C.byref(ms), _stream(stream)))
    return f.value, ms.value


# ---------------------------------------------------------------- surrogate
SURR_SIZES = (4, 256, 256, 256, 256, 81)


class MLP:
    """The f_eq surrogate (mlp_create & co.).  params: packed FP32 numpy
    vector (W_1, b_1, W_2, b_2, ...), shift/scale: feature normalisation."""

    def __init__(self, params, shift, scale, n_hidden=4, width=256, n_classes=81):
        self._params = np.ascontiguousarray(params, dtype=np.float32)
        sh = np.ascontiguousarray(shift, dtype=np.float32)
        sc = np.ascontiguousarray(scale, dtype=np.float32)
        h = P()
        _check(load().mlp_create(n_hidden, width, n_classes, _ptr(sh), _ptr(sc), _ptr(self._params),
                                 C.byref(h)))
        self.h = h
        self.n_classes = n_classes
        self.n_params = int(load().mlp_param_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            load().mlp_destroy(self.h)
            self.h = None

    __del__ = close

    def get_params(self):
        out = np.zeros(self.n_params, np.float32)
        _check(load().mlp_get_params(self.h, _ptr(out)))
        return out

    def set_params(self, params):
        p_ = np.ascontiguousarray(params, dtype=np.float32)
        _check(load().mlp_set_params(self.h, _ptr(p_)))

    def forward(self, X, out=None, stream=None):
        """X: device float32 [M, 4] -> device float32 [M, n_classes]."""
        import torch

        if out is None:
            out = torch.empty((X.shape[0], self.n_classes), dtype=torch.float32, device="cuda")
        _check(load().mlp_forward(self.h, _ptr(X), X.shape[0], _ptr(out), _stream(stream)))
        return out

    def grad(self, X, T, stream=None):
        import torch

        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        _check(load().mlp_grad(self.h, _ptr(X), _ptr(T), X.shape[0], _ptr(g), _ptr(loss),
                               _stream(stream)))
        return g, loss

    def train_step(self, X, T, lr, loss=None, stream=None):
        _check(load().mlp_train_step(self.h, _ptr(X), _ptr(T), X.shape[0], float(lr), _ptr(loss),
                                     _stream(stream)))

    def status(self):
        _check(load().mlp_status(self.h))


def bf16_gemm_tn(A, B, stream=None):
    """C = A @ B.T on the tensor cores (A [M,K], B [N,K] bf16 device tensors)."""
    import torch

    M, K = A.shape
    N = B.shape[0]
    Cm = torch.empty((M, N), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _check(load().bf16_gemm_tn(_ptr(A), _ptr(B), _ptr(Cm), M, N, K, _ptr(st), _stream(stream)))
    return Cm, st


def bf16_gemm_selftest(A, B, limit_s=0.02, stream=None):
    """Return code of bf16_gemm_selftest (MD_E_TIMEOUT when the bounded
    mbarrier waits work)."""
    import torch

    M, K = A.shape
    N = B.shape[0]
    Cm = torch.empty((M, N), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    return int(load().bf16_gemm_selftest(_ptr(A), _ptr(B), _ptr(Cm), M, N, K, _ptr(st), float(limit_s),
                                         _stream(stream)))
