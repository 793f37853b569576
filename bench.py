"""Throughput benchmark of the MDLG hot path: 2D Lennard-Jones MD with the
MDLG coarse-graining fused in, plus the f_eq stage (measured, Gaussian and
WSG equilibria and their comparison), through the C-ABI of libmdlg.so.

Workload (single large system): N = 262,144 particles at area fraction
0.0784 (L = 1620.53 sigma), T = 20, LJ with rc = 2.5 (shifted), dt = 5e-4,
FP32 cell-index + offset positions; sampling intervals Delta t_LG in
{0.05, 0.1, 0.2, 0.5, 1.0} on lattices dx in {0.5, 1, 2} (15 int32
histograms, W = 4 plus overflow), FP64 normalisation.  One bench step = 2,000
MD steps (one window of the longest interval, 38 sampling events x 3
lattices) followed by the f_eq stage for all 15 (interval, lattice) pairs.
Synthetic seeded state (square lattice + jitter, Maxwell velocities).

Output: one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload.
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
N_PART = 262_144
PHI, TEMP, DT = 0.0784, 20.0, 5e-4
LG_EVERY = (100, 200, 400, 1000, 2000)
DX = (0.5, 1.0, 2.0)
W = 4
MD_PER_STEP = 2000
BYTES_PER_PARTICLE_STEP = 40.0      # FP32 cell + offset: 20 B state read + 20 B written
L2_BYTES = 129 * 2 ** 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _profile_traffic():
    """DRAM bytes per launch of the persistent kernel from the committed ncu
    summary, scaled to one 2,000-step launch (null if absent)."""
    p = os.path.join(ROOT, "profiles", "k_md_persistent_fp32_n262144.md")
    try:
        for line in open(p):
            if line.startswith("traffic_bytes_per_2000_step_launch:"):
                v = line.split(":", 1)[1].strip()
                return None if v in ("", "null") else float(v)
    except OSError:
        pass
    return None


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


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _params(mdlg, L, prec):
    return mdlg.make_params(N_PART, L, dt=DT, precision=prec, W=W, n_equil=0, lg_every=LG_EVERY,
                            lx=tuple(int(round(L / d)) for d in DX), block_windows=1)


def _feq_stage(mdlg, sysm, torch):
    """Measured f_eq, lambda, Gaussian and WSG equilibria and their comparison
    for every (interval, lattice); returns the worst |P_MD - P_WSG| seen."""
    worst = 0.0
    for k in range(len(LG_EVERY)):
        for d in range(len(DX)):
            Pm, se, st = sysm.feq_measured(0, k, d, symmetrize=True)
            if st.n_windows == 0:
                continue
            Pd = torch.from_numpy(Pm).cuda()
            g = mdlg.feq_gaussian(st.a2, W=W)
            lam_t, rc = mdlg.wsg_lambda(st.mu2, st.mu4, allow_domain=True)
            lam = float(lam_t.item())
            wsg = mdlg.feq_wsg(st.a2, lam, W=W)
            mdlg.feq_compare(Pd, g)
            cw = mdlg.feq_compare(Pd, wsg)
            worst = max(worst, float(cw[0].item()))
    return worst


def run_ours(args):
    import torch

    from paper_2101_01160_gb300 import inputs, mdlg

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist_

        dist_.init_process_group("nccl")
        dist = dist_
    mdlg.load()
    L = inputs.box_length(N_PART, PHI)
    st = inputs.lattice_gas_state(N_PART, L, TEMP, seed=1000 + rank)
    stream = torch.cuda.current_stream()
    sysm = mdlg.System(_params(mdlg, L, mdlg.MD_FP32_CELLOFF), st.x, st.y, st.vx, st.vy, stream)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda")

    def one_step():
        sysm.step(MD_PER_STEP)
        return _feq_stage(mdlg, sysm, torch)

    for _ in range(args.warmup):
        one_step()
    sysm.sync()
    # device-timed region: per-step events, L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    worst = 0.0
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            sysm.step(MD_PER_STEP)
            ev[i][1].record(stream)
            worst = max(worst, _feq_stage(mdlg, sysm, torch))
            ev[i][2].record(stream)
        torch.cuda.synchronize()
    rc = sysm.sync()
    step_ms = sum(a.elapsed_time(c) for a, b, c in ev)
    kern_ms = [a.elapsed_time(b) for a, b, c in ev]
    t_max = step_ms
    if dist:
        t = torch.tensor([step_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
        dist.barrier()
    ms_per_step = t_max / args.steps
    value = ws * N_PART * MD_PER_STEP / (ms_per_step * 1e-3)

    # end-to-end through the C-ABI with host buffers: upload the state from
    # pinned host memory, run, read the f_eq results back
    pin = [torch.from_numpy(a).pin_memory() for a in (st.x, st.y, st.vx, st.vy)]
    host = [t.numpy() for t in pin]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 5))
    for _ in range(e2e_steps):
        sysm.set_state(*host)
        sysm.step(MD_PER_STEP)
        _feq_stage(mdlg, sysm, torch)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": ws * N_PART * MD_PER_STEP / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 4 * 8 * N_PART,
           "d2h_bytes_per_step": len(LG_EVERY) * len(DX) * (2 * (2 * W + 1) ** 2 + 8) * 8}

    peak, peak_kind = _peaks()
    kern_avg_s = (sum(kern_ms) / len(kern_ms)) * 1e-3
    achieved = BYTES_PER_PARTICLE_STEP * N_PART * MD_PER_STEP / kern_avg_s / 1e9
    info = sysm.info()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "single large system N=262144 phi=0.0784 T=20 FP32 cell+offset, "
                               "dt_lg {0.05,0.1,0.2,0.5,1.0} x dx {0.5,1,2}, W=4; "
                               "2000 MD steps + f_eq stage per step",
                   "n_particles": N_PART, "md_steps_per_step": MD_PER_STEP,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": _profile_traffic(),
                     "kernel": "k_md_persistent<float,256>", "peak_kind": peak_kind},
        "e2e": e2e,
        "gpu_launches": args.steps * (1 + 6 * len(LG_EVERY) * len(DX)),
        "clocks": clk.summary(),
        "f_eq_err_max_abs_md_vs_wsg": worst,
        "md_status": rc,
        "rebuilds": int(info.n_rebuilds),
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(st, L)
    sysm.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _oracle_sample(st, L, nsteps):
    from oracle import oracle

    lx = [int(round(L / d)) for d in DX]
    t0 = time.perf_counter()
    oracle.md_run(st.x, st.y, st.vx, st.vy, L, DT, nsteps, every=[LG_EVERY[0]], lx=lx, W=W)
    return time.perf_counter() - t0


def cpu_baseline(st, L, nsteps=200):
    dt = _oracle_sample(st, L, nsteps)
    return {"value": N_PART * nsteps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"N={N_PART} workload state, {nsteps} MD steps, binning every 100 steps on "
                      f"3 lattices; FP64 C oracle, single thread"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2101_01160_gb300 import inputs

    L = inputs.box_length(N_PART, PHI)
    st = inputs.lattice_gas_state(N_PART, L, TEMP, seed=1000)
    per = 100
    for _ in range(args.warmup):
        _oracle_sample(st, L, per)
    tot = 0.0
    for _ in range(args.steps):
        tot += _oracle_sample(st, L, per)
    ms = tot / args.steps * 1e3
    value = N_PART * per / (ms * 1e-3)
    sample = (f"N={N_PART} workload state, {per} MD steps per step, binning every 100 steps on "
              f"3 lattices; FP64 C oracle, single thread")
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": "single large system N=262144 phi=0.0784 T=20 (oracle sample)",
                   "n_particles": N_PART, "md_steps_per_step": per},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
