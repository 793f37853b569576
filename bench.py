"""Throughput benchmark of the MDLG hot path: 2D Lennard-Jones MD with the
MDLG coarse-graining fused into the step, plus the f_eq stage (measured,
Gaussian and WSG equilibria and their comparison), through the C-ABI of
libmdlg.so.

Headline workload (batched ensemble): 256 independent replicas in one
persistent launch, N log-uniform in [4096, 65536], area fraction uniform in
[0.02, 0.30], T uniform in [1, 20], per-replica seeds (square lattice +
jitter, Maxwell velocities); LJ with rc = 2.5 (shifted), dt = 5e-4, FP32
cell-index + offset positions, MDLG sampling every 400 steps (Delta t_LG =
0.2) on a lattice of spacing ~1 sigma, W = 4 (81 classes) plus overflow,
int32 histograms, FP64 normalisation.  One bench step = 400 MD steps (one
sampling window) + the batched f_eq stage for all replicas.

Also measured and reported beside it: the single large system (N = 262,144,
phi = 0.0784, T = 20, FP32, five sampling intervals x three lattices) and
the same system in plain FP64.

Output: one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on all host threads on a bounded sample of the same workload (16 of the 256
replicas, one 400-step window per step).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s incl. MDLG binning (batched FP32 vs plain FP64, 1 GB300); f_eq err"
UNIT = "particle-steps/s"
N_REP = 256
ENS_SEED = 7
DT = 5e-4
EVERY = 400
MD_PER_STEP = 400
W = 4
# Verlet skin of each replica's neighbour lists (an implementation choice:
# lists hold pairs within rc + skin and are rebuilt when a displacement
# reaches skin/2; the physics does not depend on it).  The global engine
# rebuilds every replica when any replica's displacement bound, in units of
# its own half skin, is used up, so a skin proportional to the thermal speed
# sqrt(T) lets every replica use its bound at about the same rate and gives
# the slower replicas shorter lists.  Measured on this ensemble (ms per
# 400-step bench step): one skin for all 0.6: 64.8; 0.7 sqrt(T/20), at least
# 0.2: 63.2; 0.6 sqrt(T/20), at least 0.15: 63.5; 0.6 (T/20)^0.35, at least
# 0.2: 63.5.
SKIN_HOT, SKIN_T, SKIN_MIN = 0.7, 20.0, 0.2


def skin_of(T):
    """Verlet skin of a replica at temperature T."""
    return max(SKIN_MIN, SKIN_HOT * math.sqrt(T / SKIN_T))


SKIN_TEXT = "Verlet skin 0.7 sqrt(T/20) per replica (at least 0.2)"
BYTES_PER_PARTICLE_STEP = 40.0      # FP32 cell + offset: 20 B state read + 20 B written
RESIDENT_SLAB_PARTICLES = 8192      # own particles one resident slab (one SM's shared memory) holds
L2_BYTES = 129 * 2 ** 20
# single large system (reported beside the headline)
N1, PHI1, T1 = 262_144, 0.0784, 20.0
LG1, DX1 = (100, 200, 400, 1000, 2000), (0.5, 1.0, 2.0)


def _peaks(key="hbm_gbs", fallback=6800.0):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d[key]), "measured"
    except Exception:
        return fallback, "fallback"


# DRAM traffic of one bench-step launch of the global engine's kernel on this
# workload: dram__bytes_read.sum + dram__bytes_write.sum from one ncu capture
# of k_md_persistent<float,256,1> (the launch shape the autotuner picks),
# copied here with its provenance; it is reported only for that kernel and
# launch shape, and must be re-measured when the kernel changes.
MD_TRAFFIC = {"kernel": "k_md_persistent<float,256,1>", "bytes_per_launch": 176736049050,
              "source": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                        "over every launch of 'bench.py --steps 2 --warmup 3 --no-cpu-baseline "
                        "--no-variants' (one pass), mean of the five 400-step launches of warm-up "
                        "and timed region (Verlet skin 0.7 sqrt(T/20) per replica, at least 0.2): "
                        "127.7 GB read + 49.0 GB written, 77.4 B per particle-step"}


def _cpu_model():
    """CPU model of this host as the OS reports it (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part", "hardware")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _flops_per_particle_step(ens, skin=None, rc=2.5):
    """Algorithmic flops of one particle-step of the list-based LJ step
    (full neighbour lists, each pair evaluated from both sides), averaged
    over the particles of the ensemble: per listed pair the pair vector and
    r^2 (5 flops), per pair within rc the force (13 more: 1/r^2, s^6, the
    force factor and two multiply-adds), per particle the two half kicks,
    the drift and the speed bound (16).  Mean counts from the density:
    pi rc^2 n pairs within rc, pi (rc + skin)^2 n listed (skin: one for all,
    else each replica's skin_of(T))."""
    tot, num = 0.0, 0.0
    for (n, L, *rest) in ens:
        dens = n / (L * L)
        within = np.pi * rc * rc * dens
        sk = skin if skin is not None else skin_of(rest[1])
        listed = np.pi * (rc + sk) ** 2 * dens
        num += n * (5.0 * listed + 13.0 * within + 16.0)
        tot += n
    return num / tot


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def ensemble(seed_offset=0, reps=None):
    """Per-replica parameters and initial states of the batched ensemble."""
    from paper_2101_01160_gb300 import inputs

    Ns, phis, Ts = inputs.ensemble_params(N_REP, seed=ENS_SEED + seed_offset)
    out = []
    for r in (range(N_REP) if reps is None else reps):
        n = int(Ns[r])
        L = inputs.box_length(n, float(phis[r]))
        st = inputs.lattice_gas_state(n, L, float(Ts[r]), seed=100_000 * seed_offset + r)
        out.append((n, L, float(phis[r]), float(Ts[r]), st))
    return out


WORKLOAD = (f"batched ensemble: {N_REP} replicas, N log-uniform [4096,65536], phi U[0.02,0.30], "
            f"T U[1,20], FP32 cell+offset, dt 5e-4, {SKIN_TEXT}, sampling every 400 steps "
            "(dt_lg 0.2) on dx~1, W=4; 400 MD steps + batched f_eq stage per step")


def _ensemble_particles(seed_offset=0):
    """Total particle count of the ensemble (no states built)."""
    from paper_2101_01160_gb300 import inputs

    Ns, _, _ = inputs.ensemble_params(N_REP, seed=ENS_SEED + seed_offset)
    return int(sum(int(n) for n in Ns))


def _ens_params(mdlg, ens, prec):
    return [mdlg.make_params(n, L, dt=DT, precision=prec, W=W, n_equil=0, lg_every=(EVERY,),
                             lx=(int(round(L)),), skin=skin_of(T)) for (n, L, _, T, _) in ens]


def _time_variant(mdlg, torch, params, st, md_steps, reps=3):
    """Device time of md_step(md_steps) launches on one system."""
    s = mdlg.System(params, st.x, st.y, st.vx, st.vy)
    s.autotune(100)
    s.step(md_steps)
    s.sync()
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.step(md_steps)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    s.sync()
    s.close()
    m = float(np.median(ms))
    return {"value": params.n * md_steps / (m * 1e-3), "ms_per_launch": m, "md_steps": md_steps}


def _time_surrogate(mdlg, torch, n=1 << 20, reps=20):
    """Fused f_eq-surrogate forward pass (4 -> 256 x4 SiLU -> 81 softmax,
    BF16 tensor cores) on n query points; random-initialised weights of the
    trained architecture (the flop count does not depend on the values)."""
    from paper_2101_01160_gb300 import inputs, surrogate

    model = surrogate.new_model(0)
    X = torch.from_numpy(inputs.surrogate_queries(n, 3, lo=(0.02, 1.0, 0.05, 1.0),
                                                  hi=(0.30, 20.0, 0.2, 4.0))).cuda()
    out = torch.empty((n, model.n_classes), dtype=torch.float32, device="cuda")
    m = _time_queued(torch, lambda: model.forward(X, out=out), reps)
    model.status()
    sizes = mdlg.SURR_SIZES
    flop = 2.0 * sum(a * b for a, b in zip(sizes[:-1], sizes[1:])) * n
    peak, kind = _peaks("bf16_tflops", 1900.0)
    tf = flop / (m * 1e-3) / 1e12
    return {"queries": n, "ms_per_launch": m, "queries_per_s": n / (m * 1e-3), "tflops": tf,
            "bf16_peak_tflops": peak, "peak_kind": kind, "frac": tf / peak,
            "kernel": "k_mlp_fused", "workload": "1,048,576 queries uniform in the training box"}


def _time_surrogate_training(mdlg, torch, batch=8192, reps=20):
    """One Adam training step of the f_eq surrogate (forward, KL loss and
    backward GEMMs on the tensor cores, Adam update) on a batch of synthetic
    queries and target distributions; algorithmic flops 3x the forward's per
    sample (forward, input gradient, weight gradient)."""
    from paper_2101_01160_gb300 import inputs, surrogate

    model = surrogate.new_model(1)
    X = torch.from_numpy(inputs.surrogate_queries(batch, 5, lo=(0.02, 1.0, 0.05, 1.0),
                                                  hi=(0.30, 20.0, 0.2, 4.0))).cuda()
    g = torch.Generator(device="cuda")
    g.manual_seed(6)
    T = torch.rand((batch, model.n_classes), device="cuda", generator=g)
    T = (T / T.sum(dim=1, keepdim=True)).contiguous()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    for _ in range(3):
        model.train_step(X, T, 1e-4, loss=loss)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        model.train_step(X, T, 1e-4, loss=loss)
    e1.record()
    torch.cuda.synchronize()
    model.status()
    ms = e0.elapsed_time(e1) / reps
    sizes = mdlg.SURR_SIZES
    flop = 3 * 2.0 * sum(a * b for a, b in zip(sizes[:-1], sizes[1:])) * batch
    peak, kind = _peaks("bf16_tflops", 1900.0)
    tf = flop / (ms * 1e-3) / 1e12
    return {"batch": batch, "ms_per_step": ms, "samples_per_s": batch / (ms * 1e-3), "tflops": tf,
            "bf16_peak_tflops": peak, "peak_kind": kind, "frac": tf / peak,
            "workload": "Adam steps on 8192 synthetic (query, distribution) pairs, steps queued back to back"}


def _time_queued(torch, fn, reps=20):
    """Device time of one launch of fn with a cold L2: reps x (256 MB L2
    flush + fn) queued back to back between two CUDA events, less reps
    flushes alone, over reps.  The queue keeps the GPU ahead of the host, so
    the host's call overhead is not counted."""
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def span(with_fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            flush.zero_()
            if with_fn:
                fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    for _ in range(3):
        fn()
    span(True)
    both = min(span(True) for _ in range(3))
    alone = min(span(False) for _ in range(3))
    return max(both - alone, 0.0) / reps


def _time_disp_hist(mdlg, torch, n=1 << 24, reps=20):
    """Displacement-PDF histogram (Sec. 3(b), Fig. 2) of a synthetic FP32
    snapshot pair of n particles (400 MB, above L2); algorithmic traffic
    24 B per particle (two snapshots of cell + two FP32 offsets)."""
    from paper_2101_01160_gb300 import inputs

    ncell = 2160
    h = float(np.float32(6482.12 / ncell))
    s = inputs.random_celloff_snapshots(n, ncell, h, seed=5, max_step=6.0)
    arrs = [torch.from_numpy(s[k]).cuda() for k in ("cell0", "ox0", "oy0", "cell1", "ox1", "oy1")]
    m = _time_queued(torch, lambda: mdlg.disp_hist(*arrs, ncell, h, 0.05, 512), reps)
    peak, kind = _peaks()
    gbs = 24.0 * n / (m * 1e-3) / 1e9
    return {"particles": n, "ms_per_launch": m, "gbs": gbs, "peak_gbs": peak, "peak_kind": kind,
            "frac": gbs / peak, "kernel": "k_disp_hist", "bytes_per_particle": 24,
            "workload": "synthetic FP32 snapshot pair, 16.8M particles, 512 bins of 0.05 sigma"}


def _time_local_fields(mdlg, torch, reps=20):
    """Local MDLG fields (Sec. 2, Eqs. n_i and mdlg_evolution) of a synthetic
    ensemble snapshot pair: 64 replicas of the standard system's box (N =
    99,856, L = 1000) in one call, on Table 1's lx = 250 lattice, W = 4.
    Algorithmic traffic: 24 B per
    particle for the occupation numbers (two FP32 snapshots; the 20 MB field
    stays in L2), 12 B per field entry for the collision operator (two int32
    fields read, one written).  L2 is flushed before every launch."""
    from paper_2101_01160_gb300 import inputs

    n, ncell, lx, W = 64 * 99_856, 333, 250, 4
    h = float(np.float32(1000.0 / ncell))
    s = inputs.random_celloff_snapshots(n, ncell, h, seed=77, max_step=4.0, lattice_dx=ncell * h / lx)
    d = [torch.from_numpy(s[k]).cuda() for k in ("cell0", "ox0", "oy0", "cell1", "ox1", "oy1")]
    field, ovf = mdlg.site_occupation(*d, ncell, h, lx, W)
    f2, _ = mdlg.site_occupation(*d, ncell, h, lx, W)
    xi = torch.empty_like(field)
    lib = mdlg.load()
    out = {
        "occupation": _time_queued(torch, lambda: mdlg.site_occupation(*d, ncell, h, lx, W, field=field, ovf=ovf), reps),
        # the C entry point directly, writing into a preallocated Xi field
        "collision": _time_queued(torch, lambda: lib.mdlg_collision(mdlg._ptr(field), mdlg._ptr(f2), lx, W, 1.0,
                                                                    mdlg._ptr(xi), None, None), reps),
    }
    peak, kind = _peaks()
    entries = (2 * W + 1) ** 2 * lx * lx
    g_occ = 24.0 * n / (out["occupation"] * 1e-3) / 1e9
    g_col = 12.0 * entries / (out["collision"] * 1e-3) / 1e9
    return {"particles": n, "field_entries": entries,
            "occupation": {"kernel": "k_site_occupation", "ms_per_launch": out["occupation"], "gbs": g_occ,
                           "frac": g_occ / peak, "bytes_per_particle": 24},
            "collision": {"kernel": "k_collision", "ms_per_launch": out["collision"], "gbs": g_col,
                          "frac": g_col / peak, "bytes_per_entry": 12},
            "peak_gbs": peak, "peak_kind": kind,
            "workload": "synthetic FP32 ensemble snapshot pair, 64 x 99,856 particles, L = 1000, lx = 250, W = 4"}


def run_profile_case(args):
    """Small cases for ncu captures (not a bench line): res16 = the first 16
    replicas of the batched ensemble (about 360k particles) on the
    shared-memory-resident engine, one 400-step launch then three 100-step
    launches; md64 = the first 64
    replicas of the batched ensemble (about 1.4M particles, > L2), fixed
    launch shape (256 threads, 1 chunk per thread, global staging with the
    full-occupancy register budget, as the autotuner picks for the bench), two
    400-step warm-up launches then three 100-step launches; mlp = three fused
    surrogate forward passes on 1M queries; train = four surrogate training
    steps on 8192 synthetic samples; disp = eight displacement-PDF
    histograms of a 16.8M-particle snapshot pair; local = the occupation and
    collision kernels of the local fields on a 6.4M-particle ensemble snapshot
    pair (two occupation calls, then three occupation + collision pairs)."""
    import torch

    from paper_2101_01160_gb300 import mdlg

    mdlg.load()
    if args.profile_case == "res16":
        ens = ensemble(reps=range(16))
        cat = [np.concatenate([getattr(e[4], f) for e in ens]) for f in ("x", "y", "vx", "vy")]
        s = mdlg.System(_ens_params(mdlg, ens, mdlg.MD_FP32_CELLOFF), *cat)
        s.tune(0, 0, 4)
        s.step(MD_PER_STEP)
        for _ in range(3):
            s.step(100)
        s.sync()
        print(json.dumps({"profile_case": "res16", "n_particles": int(sum(e[0] for e in ens)),
                          "rebuilds": int(s.info().n_rebuilds)}))
        s.close()
    elif args.profile_case == "train":
        from paper_2101_01160_gb300 import inputs, surrogate

        model = surrogate.new_model(1)
        B = 8192
        X = torch.from_numpy(inputs.surrogate_queries(B, 5, lo=(0.02, 1.0, 0.05, 1.0),
                                                      hi=(0.30, 20.0, 0.2, 4.0))).cuda()
        g = torch.Generator(device="cuda")
        g.manual_seed(6)
        T = torch.rand((B, model.n_classes), device="cuda", generator=g)
        T = (T / T.sum(dim=1, keepdim=True)).contiguous()
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        for _ in range(4):
            model.train_step(X, T, 1e-4, loss=loss)
        torch.cuda.synchronize()
        model.status()
        print(json.dumps({"profile_case": "train", "batch": B, "loss": float(loss.item())}))
    elif args.profile_case == "md64":
        ens = ensemble(reps=range(64))
        cat = [np.concatenate([getattr(e[4], f) for e in ens]) for f in ("x", "y", "vx", "vy")]
        s = mdlg.System(_ens_params(mdlg, ens, mdlg.MD_FP32_CELLOFF), *cat)
        s.tune(256, 1, 3)
        for _ in range(2):
            s.step(MD_PER_STEP)
        for _ in range(3):
            s.step(100)
        s.sync()
        print(json.dumps({"profile_case": "md64", "n_particles": int(sum(e[0] for e in ens)),
                          "rebuilds": int(s.info().n_rebuilds)}))
        s.close()
    elif args.profile_case == "disp":
        r = _time_disp_hist(mdlg, torch, reps=3)
        print(json.dumps({"profile_case": "disp", **r}))
    elif args.profile_case == "local":
        from paper_2101_01160_gb300 import inputs

        n, ncell, lx, W = 64 * 99_856, 333, 250, 4
        h = float(np.float32(1000.0 / ncell))
        sn = inputs.random_celloff_snapshots(n, ncell, h, seed=77, max_step=4.0, lattice_dx=ncell * h / lx)
        d = [torch.from_numpy(sn[k]).cuda() for k in ("cell0", "ox0", "oy0", "cell1", "ox1", "oy1")]
        field, ovf = mdlg.site_occupation(*d, ncell, h, lx, W)
        f2, _ = mdlg.site_occupation(*d, ncell, h, lx, W)
        for _ in range(3):
            mdlg.site_occupation(*d, ncell, h, lx, W, field=field, ovf=ovf)
            mdlg.collision(field, f2, W)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "local", "particles": n, "field_entries": int(field.numel())}))
    else:
        r = _time_surrogate(mdlg, torch, reps=3)
        print(json.dumps({"profile_case": "mlp", **r}))


def run_ours(args):
    import torch

    from paper_2101_01160_gb300 import inputs, mdlg, sharding

    ws, rank, local = sharding.world()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist_

        dist_.init_process_group("nccl")
        dist = dist_
    mdlg.load()
    ens = ensemble(seed_offset=sharding.seed_offset(rank))
    ntot = sum(e[0] for e in ens)
    cat = [np.concatenate([getattr(e[4], f) for e in ens]) for f in ("x", "y", "vx", "vy")]
    stream = torch.cuda.current_stream()
    sysm = mdlg.System(_ens_params(mdlg, ens, mdlg.MD_FP32_CELLOFF), *cat, stream=stream)
    nb = (2 * W + 1) ** 2
    feq_dev = torch.empty((N_REP, 3 * nb + mdlg.FEQB_STATS), dtype=torch.float64, device="cuda")
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda")
    shape = sysm.autotune(100)      # launch shape (untimed set-up; real MD steps)
    peaks = measured_alu_peaks(mdlg)

    for _ in range(args.warmup):
        sysm.step(MD_PER_STEP)
        mdlg.feq_batch(sysm, 0, 0, True, out=feq_dev)
    sysm.sync()
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            sysm.step(MD_PER_STEP)
            ev[i][1].record(stream)
            mdlg.feq_batch(sysm, 0, 0, True, out=feq_dev)
            ev[i][2].record(stream)
        torch.cuda.synchronize()
    sysm.sync()
    step_ms = sum(a.elapsed_time(c) for a, b, c in ev)
    kern_ms = [a.elapsed_time(b) for a, b, c in ev]
    # whole job: particle-steps summed over ranks / slowest rank's timed region
    ps_all, t_max = sharding.aggregate(dist, ntot * MD_PER_STEP * args.steps, step_ms)
    ms_per_step = t_max / args.steps
    value = ps_all / (t_max * 1e-3)
    stats = feq_dev[:, 3 * nb:].cpu().numpy()
    fd = feq_dev.cpu().numpy()
    dw = np.abs(fd[:, :nb] - fd[:, 2 * nb:3 * nb])
    r_w, i_w = np.unravel_index(int(np.argmax(dw)), dw.shape)
    dg = np.abs(fd[:, :nb] - fd[:, nb:2 * nb])
    r_g, i_g = np.unravel_index(int(np.argmax(dg)), dg.shape)
    # 3 sigma of the measured value there: batch means over blocks of windows
    _, se_w, _ = sysm.feq_measured(int(r_w), 0, 0, symmetrize=True)
    _, se_g, _ = sysm.feq_measured(int(r_g), 0, 0, symmetrize=True)
    feq_err = {"max_abs_md_vs_wsg": float(dw[r_w, i_w]), "max_abs_md_vs_wsg_3sigma": float(3 * se_w[i_w]),
               "max_abs_md_vs_gauss": float(dg[r_g, i_g]), "max_abs_md_vs_gauss_3sigma": float(3 * se_g[i_g]),
               "at": {"wsg": [int(r_w), int(i_w)], "gauss": [int(r_g), int(i_g)]},
               "median_kl_md_wsg": float(np.median(stats[:, 7])),
               "median_kl_md_gauss": float(np.median(stats[:, 5])),
               "windows": int(stats[0, 8]),
               "sigma": "batch means over 32 blocks of windows, symmetric-set averages"}
    # the same bars from the block bootstrap of every replica (200 resamples
    # of its error-bar blocks of windows), and the share of (replica, class)
    # entries whose model deviation lies within them
    sb = mdlg.feq_bootstrap(sysm, 0, 0, symmetrize=True, n_resamples=200, seed=11)
    ok = sb > 0
    feq_err["bootstrap"] = {
        "max_abs_md_vs_wsg_3sigma": float(3 * sb[r_w, i_w]),
        "max_abs_md_vs_gauss_3sigma": float(3 * sb[r_g, i_g]),
        "frac_within_3sigma": {"wsg": float(np.mean(dw[ok] <= 3 * sb[ok])),
                               "gauss": float(np.mean(dg[ok] <= 3 * sb[ok]))},
        "resamples": 200}

    # end to end through the C-ABI with host buffers: every step uploads the
    # (equilibrated) state from pinned host memory, runs one window and reads
    # the f_eq stage back.  The upload of the next step's state runs on a copy
    # stream while the current step computes (the first one before it), into
    # a device staging buffer that md_set_state reads; all copies are inside
    # the timed region.
    pin = [torch.from_numpy(a).pin_memory() for a in sysm.get_state()]
    stage = [torch.empty_like(t, device="cuda") for t in pin]
    copy_stream = torch.cuda.Stream()
    e2e_steps = max(1, min(args.steps, 5))

    def upload():
        with torch.cuda.stream(copy_stream):
            for d, h in zip(stage, pin):
                d.copy_(h, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(copy_stream)
        return ev

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev = upload()
    for k in range(e2e_steps):
        ev.synchronize()
        sysm.set_state(*stage)
        if k + 1 < e2e_steps:
            ev = upload()
        sysm.step(MD_PER_STEP)
        mdlg.feq_batch(sysm, 0, 0, True)
    torch.cuda.synchronize()
    e2e_ps, e2e_ms = sharding.aggregate(dist, ntot * MD_PER_STEP * e2e_steps,
                                        (time.perf_counter() - t0) * 1e3)
    e2e = {"value": e2e_ps / (e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": 4 * 8 * ntot,
           "d2h_bytes_per_step": N_REP * (3 * nb + mdlg.FEQB_STATS) * 8}
    info = sysm.info()
    sysm.close()

    peak, peak_kind = _peaks()
    variants = {}
    if not args.no_variants and rank == 0:
        L1 = inputs.box_length(N1, PHI1)
        st1 = inputs.lattice_gas_state(N1, L1, T1, seed=1000)
        lx1 = tuple(int(round(L1 / d)) for d in DX1)
        for name, prec in (("single_system_fp32", mdlg.MD_FP32_CELLOFF),
                           ("plain_fp64", mdlg.MD_FP64)):
            p = mdlg.make_params(N1, L1, dt=DT, precision=prec, W=W, lg_every=LG1, lx=lx1)
            variants[name] = _time_variant(mdlg, torch, p, st1, 2000)
            variants[name]["workload"] = ("N=262144 phi=0.0784 T=20, dt_lg {0.05..1.0} x dx "
                                          "{0.5,1,2}, one 2000-step launch")
        v64 = variants["plain_fp64"]
        f64 = _flops_per_particle_step([(N1, L1)], skin=0.5)
        ach = f64 * v64["value"] / 1e12
        hbm_ps = peak * 1e9 / 64.0                      # 32 B read + 32 B written per particle-step
        alu_ps = peaks["fp64_tflops"] * 1e12 / f64
        v64["roofline"] = {"bound": "fp64_alu" if alu_ps < hbm_ps else "hbm", "achieved": ach,
                           "peak": peaks["fp64_tflops"], "unit": "TFLOP/s", "frac": ach / peaks["fp64_tflops"],
                           "flops_per_particle_step": f64, "hbm_frac": 64.0 * v64["value"] / (peak * 1e9),
                           "bound_particle_steps_per_s": min(hbm_ps, alu_ps),
                           "frac_of_bound": v64["value"] / min(hbm_ps, alu_ps)}
        variants["equal_accuracy"] = _equal_accuracy(mdlg, torch)
        variants["surrogate_inference"] = _time_surrogate(mdlg, torch)
        variants["surrogate_training"] = _time_surrogate_training(mdlg, torch)
        variants["disp_hist"] = _time_disp_hist(mdlg, torch)
        variants["local_fields"] = _time_local_fields(mdlg, torch)

    kern_avg_s = (sum(kern_ms) / len(kern_ms)) * 1e-3
    achieved = BYTES_PER_PARTICLE_STEP * ntot * MD_PER_STEP / kern_avg_s / 1e9
    kname = ("k_md_resident" if shape[2] == 4 else
             f"k_md_persistent<float,{shape[0]},{int(shape[2] == 3)}>")
    traffic = MD_TRAFFIC["bytes_per_launch"] if kname == MD_TRAFFIC["kernel"] else None
    fpps = _flops_per_particle_step(ens)
    alu = {"bound": "alu", "achieved": fpps * ntot * MD_PER_STEP / kern_avg_s / 1e12,
           "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
           "flops_per_particle_step": fpps, "peak_kind": "measured FP32 FMA throughput (this run)"}
    alu["frac"] = alu["achieved"] / alu["peak"]
    # composite bound of the ensemble: per replica the larger of its state
    # traffic over the HBM bandwidth and its flops over the FP32 FMA peak,
    # a replica that fits one SM's shared memory for a whole launch (the
    # resident engine's slab capacity) counted with no HBM traffic
    t_bound = 0.0
    for e in ens:
        n = e[0]
        b = 0.0 if n <= RESIDENT_SLAB_PARTICLES else BYTES_PER_PARTICLE_STEP * n * MD_PER_STEP
        f = _flops_per_particle_step([e]) * n * MD_PER_STEP
        t_bound += max(b / (peak * 1e9), f / (peaks["fp32_tflops"] * 1e12))
    composite = {"bound_ms": t_bound * 1e3, "kernel_ms": kern_avg_s * 1e3, "frac": t_bound / kern_avg_s,
                 "resident_below_particles": RESIDENT_SLAB_PARTICLES,
                 "how": "sum over replicas of max(40 B x particle-steps / HBM, flops / FP32 FMA peak)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "n_particles": ntot, "md_steps_per_step": MD_PER_STEP,
                   "l2": "flushed between timed steps (256 MB write)",
                   "launch_shape": {"block_threads": shape[0], "per_thread": shape[1],
                                    "staging": {1: "shared", 2: "global",
                                                3: "global, full-occupancy registers",
                                                4: "shared-memory-resident slabs"}[shape[2]]},
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": kname,
                     "peak_kind": peak_kind,
                     "bytes_per_particle_step": BYTES_PER_PARTICLE_STEP},
        # the same kernel against the measured FP32 FMA rate (its arithmetic)
        "roofline_alu": alu,
        "roofline_composite": composite,
        "peaks_measured": peaks,
        "e2e": e2e,
        # per step: the persistent MD launch and the f_eq stage's three
        # (moments and lambda, WSG terms split over CTAs, the rest)
        "gpu_launches": args.steps * 4,
        "clocks": clk.summary(),
        "f_eq_err": feq_err,
        "variants": variants,
        "rebuilds": int(info.n_rebuilds),
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def measured_alu_peaks(mdlg):
    """FP32 and FP64 fused multiply-add throughput of this GPU, measured now
    (mdlg_fma_peak: the full resident grid, 8 independent chains a thread)."""
    f32, _ = mdlg.fma_peak(0, 1 << 22)
    f64, _ = mdlg.fma_peak(1, 1 << 16)
    return {"fp32_tflops": f32 / 1e12, "fp64_tflops": f64 / 1e12,
            "how": "mdlg_fma_peak: FFMA/DFMA chains over the full resident grid, CUDA events"}


def _equal_accuracy(mdlg, torch, windows=32, target=1e-4):
    """Time each path needs to measure P0 (the zero-displacement class of
    f_eq, Eq. theory_feq) to the same standard error at the same (phi, T,
    dt_lg, dx): phi = 0.0784, T = 20, dt_lg = 0.2 (400 steps of 5e-4), dx ~ 1.
    Batched FP32: 64 replicas of 16,384 particles (one launch, the autotuned
    engine); error of the replica mean from the spread over replicas.  Plain
    FP64: one system of 262,144 particles; error by batch means over the
    windows.  Both sample `windows` windows after 2,000 untimed steps; the
    time to reach `target` scales the timed run by (sigma / target)^2."""
    from paper_2101_01160_gb300 import inputs

    c0 = (2 * W + 1) ** 2 // 2
    out = {"target_sigma_p0": target, "windows": windows, "phi": PHI1, "T": T1, "dt_lg": 0.2}
    neq = 2000

    def timed(sysm, steps):
        sysm.step(neq)
        sysm.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sysm.step(steps)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    # batched FP32
    R, n = 64, 16_384
    L = inputs.box_length(n, PHI1)
    states = [inputs.lattice_gas_state(n, L, T1, seed=5000 + r) for r in range(R)]
    cat = [np.concatenate([getattr(st, f) for st in states]) for f in ("x", "y", "vx", "vy")]
    p = mdlg.make_params(n, L, dt=DT, precision=mdlg.MD_FP32_CELLOFF, W=W, n_equil=neq, lg_every=(EVERY,),
                         lx=(int(round(L)),), skin=skin_of(T1))
    s = mdlg.System([p] * R, *cat)
    shape = s.autotune(50)
    s.close()
    s = mdlg.System([p] * R, *cat)
    s.tune(*shape)
    t = timed(s, windows * EVERY)
    p0 = np.array([s.feq_measured(r, 0, 0)[0][c0] for r in range(R)])
    s.close()
    sig = float(p0.std(ddof=1) / np.sqrt(R))
    out["batched_fp32"] = {"replicas": R, "n": n, "seconds": t, "p0": float(p0.mean()), "sigma_p0": sig,
                           "seconds_to_target": t * (sig / target) ** 2, "launch_shape": list(shape)}
    # plain FP64
    L1 = inputs.box_length(N1, PHI1)
    st = inputs.lattice_gas_state(N1, L1, T1, seed=1000)
    p = mdlg.make_params(N1, L1, dt=DT, precision=mdlg.MD_FP64, W=W, n_equil=neq, lg_every=(EVERY,),
                         lx=(int(round(L1)),))
    s = mdlg.System(p, st.x, st.y, st.vx, st.vy)
    s.autotune(50)
    t = timed(s, windows * EVERY)
    P, se, _ = s.feq_measured(0, 0, 0)
    s.close()
    sig = float(se[c0])
    out["plain_fp64"] = {"n": N1, "seconds": t, "p0": float(P[c0]), "sigma_p0": sig,
                         "seconds_to_target": t * (sig / target) ** 2}
    out["fp64_over_fp32_time"] = out["plain_fp64"]["seconds_to_target"] / out["batched_fp32"]["seconds_to_target"]
    return out


SAMPLE_REPS = list(range(0, N_REP, 16))     # 16 replicas spread over the draw order


def _oracle_threads(reps, nsteps, threads):
    """The oracle over the given replicas of the ensemble, one replica per
    host thread at a time (the C oracle runs with the GIL released); returns
    (particle-steps, seconds)."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle

    ens = sorted(ensemble(reps=reps), key=lambda e: -e[0])   # largest first: fuller threads
    oracle.lib()

    def one(e):
        n, L, _, _, st = e
        oracle.md_run(st.x, st.y, st.vx, st.vy, L, DT, nsteps, every=[EVERY], lx=[int(round(L))], W=W)
        return n * nsteps

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        ps = sum(ex.map(one, ens))
    return ps, time.perf_counter() - t0


def _sample_desc(reps, nsteps, threads):
    n = sum(e[0] for e in ensemble(reps=reps))
    return (f"replicas {reps} of the batched ensemble ({n} particles), {nsteps} MD steps each "
            f"(one sampling window), FP64 C oracle, {threads} host threads, one replica per thread at a time")


def cpu_baseline():
    cores = os.cpu_count() or 1
    ps, dt = _oracle_threads(SAMPLE_REPS, MD_PER_STEP, cores)
    ps1, dt1 = _oracle_threads(SAMPLE_REPS[:2], MD_PER_STEP, 1)
    return {"value": ps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": _sample_desc(SAMPLE_REPS, MD_PER_STEP, cores), "cpu_model": _cpu_model(),
            "single_thread": {"value": ps1 / dt1, "sample": _sample_desc(SAMPLE_REPS[:2], MD_PER_STEP, 1)}}


def run_reference(args):
    from paper_2101_01160_gb300 import sharding

    ws, rank, _ = sharding.world()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        _oracle_threads(SAMPLE_REPS, MD_PER_STEP // 4, cores)
    ps_tot, tot = 0, 0.0
    for _ in range(args.steps):
        ps, dt = _oracle_threads(SAMPLE_REPS, MD_PER_STEP, cores)
        ps_tot += ps
        tot += dt
    value = ps_tot / tot
    ms = tot / args.steps * 1e3
    n_sample = sum(e[0] for e in ensemble(reps=SAMPLE_REPS))
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "n_particles": _ensemble_particles(),
                   "md_steps_per_step": MD_PER_STEP, "parallelism": f"{cores} host threads",
                   "sample": {"replicas": SAMPLE_REPS, "n_particles": n_sample,
                              "md_steps_per_step": MD_PER_STEP}},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": _sample_desc(SAMPLE_REPS, MD_PER_STEP, cores), "cpu_model": _cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--profile-case", choices=["md64", "res16", "mlp", "train", "disp", "local"], default=None,
                    help="run a small case for ncu captures instead of the bench")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
