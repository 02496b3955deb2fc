#!/usr/bin/env python
"""Benchmark: wall seconds per ESDIRK3 physical step with every implicit stage
driven to a 1e-8 relative residual drop, plus DOF-sweeps/s, in three
arithmetics of the element-Jacobi P-multigrid V-cycle:

  mixed         FP32 blocks; the smoothing sweeps' residual-and-update in
                double-word (float-float) arithmetic on every level; the
                finest level's residual (stopping norm, restricted defect)
                in binary64.  The headline value.
  mixed_bf16    as mixed, with BF16 block inverses applied with FP32
                accumulation.
  mixed_f64res  FP32 blocks, binary64 residual everywhere.
  fp64          FP64 blocks, binary64 residual everywhere.
  nk_pmg        as mixed, with every stage solved by Newton-Krylov (FGMRES,
                difference Jacobian, one FAS V-cycle as the preconditioner)
                instead of pseudo-transient continuation.

Workload (default "c2"): isentropic vortex, Ma_inf = 0.005, periodic
[0,10]^2, 64x64 straight quads, P{3-2-1-0}, I{5-10-20-40}, ESDIRK3,
dt = 0.1, dtau 0.01 -> 10, smoother refresh every 10 pseudo-iterations, the
residual norm with each equation divided by its free-stream convective flux
scale.  The vortex is advanced by consecutive physical steps from the
analytic state: W untimed warm-up steps, then K timed steps of the mixed leg;
the other legs time the first min(K, --other-steps) of the same physical
steps from the same warmed state, and the line reports how far their states
are from the mixed leg's after those steps.  Inputs are synthetic and
resident in HBM when a timed step starts.  L2 is flushed before every timed
step by writing a 256 MiB buffer.

One JSON line is printed by rank 0.  Under torchrun (N > 1) every rank runs
an independent replica (weak scaling, no data-path collective).
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

METRIC = "wall s per ESDIRK step to 1e-8 residual drop, mixed vs FP64 V-cycle; DOF-sweeps/s"
VCYCLE_FILE = os.path.join(ROOT, "profiles", "c2_step_vcycles.json")

WORKLOADS = {
    "c2": dict(name="2D Euler isentropic vortex, Ma_inf=0.005, periodic [0,10]^2, 64x64 straight quads, "
                    "P{3-2-1-0} (64 DOFs/elem), I{5-10-20-40}, ESDIRK3 dt=0.1, consecutive steps from the "
                    "analytic state, each stage to a 1e-8 relative drop of the free-stream-scaled norm",
               n=64, levels=[3, 2, 1, 0], smooth=[5, 10, 20, 40], dt=0.1),
    "c1": dict(name="2D Euler isentropic vortex, Ma_inf=0.005, periodic [0,10]^2, 8x8 straight quads, "
                    "P{2-1-0} (36 DOFs/elem), I{5-10-20}, ESDIRK3 dt=0.1, consecutive steps from the analytic "
                    "state, each stage to a 1e-8 relative drop of the free-stream-scaled norm",
               n=8, levels=[2, 1, 0], smooth=[5, 10, 20], dt=0.1),
}

def dof_sweeps_per_vcycle(E, levels, smooth):
    """sum_l DOF_l x sweeps_l: 2 n_l on every level but the coarsest, n_L there."""
    tot = 0
    for l, (P, n) in enumerate(zip(levels, smooth)):
        sweeps = n if l == len(levels) - 1 else 2 * n
        tot += 4 * E * (P + 1) ** 2 * sweeps
    return tot


# ------------------------------------------------ algorithmic work per launch
def apply_bytes(P, E, wbytes):
    n = 4 * (P + 1) ** 2
    return E * (wbytes * n * n + 16 * n + 24 * n)


def apply_flops(P, E):
    n = 4 * (P + 1) ** 2
    return E * 2 * n * n


# ------------------------------------------------------------------ helpers
# The translation units of the kernels whose ncu counters profiles/ holds (the
# double-word sweep, face-flux and residual-and-update kernels) and the device
# headers they include.
FINGERPRINT_FILES = ("k_fused.cu", "k_residual.cu", "k_volume_dw.cu", "sweep_common.cuh", "dword.cuh",
                     "physics.cuh", "physics_dw.cuh", "tma.cuh", "pmg_internal.h")


def csrc_fingerprint(src=None):
    """Hash of the recorded kernels' sources (FINGERPRINT_FILES) with comments
    and blank space removed; other kernels' files, host-only files (api.cu,
    host_tables.cpp) and comments do not change those kernels' counters."""
    import hashlib
    import re
    src = src or os.path.join(ROOT, "paper_1908_03972_gb300", "csrc")
    h = hashlib.sha256()
    for f in FINGERPRINT_FILES:
        h.update(f.encode())
        with open(os.path.join(src, f)) as fh:
            text = re.sub(r"/\*.*?\*/", "", re.sub(r"//[^\n]*", "", fh.read()), flags=re.S)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier_max(value, world, device):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------ reference arm
def cpu_model():
    """CPU model name of the host (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample(wl, n_ref, n_plain, threads=1):
    """Time the FP64 CPU oracle on one V-cycle with smoother rebuild and one
    without, on the full workload, with `threads` host threads on its element
    loops, and scale to one step (n_ref rebuilding and n_plain plain V-cycles)."""
    import oracle as O
    from paper_1908_03972_gb300 import workloads as W
    used = O.set_threads(threads)
    nodes, nbr = W.periodic_box(wl["n"], wl["n"], Ng=1)
    orc = O.Oracle(nodes, nbr, 1, wl["levels"], wl["smooth"], tol=1e-8, res_scale=W.freestream_scales(0.005))
    q = W.isentropic_vortex(orc.coords())
    A, b, c = O.esdirk3()
    dt = wl["dt"]
    odt = A[1, 1] * dt
    R = orc.residual(q)
    rho = q[0] / q[3]
    qc = np.stack([rho, rho * q[1], rho * q[2], rho * (q[3] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2))])
    orc.set_stage((qc + dt * A[1, 0] * R) / odt, odt)
    t0 = time.perf_counter()
    q1 = orc.vcycle(q, 0.01, refresh=True)
    t1 = time.perf_counter()
    orc.vcycle(q1, 0.01, refresh=False)
    t2 = time.perf_counter()
    O.set_threads(1)
    t_ref, t_plain = t1 - t0, t2 - t1
    return dict(t_vcycle_refresh=t_ref, t_vcycle=t_plain, s_per_step=n_ref * t_ref + n_plain * t_plain,
                threads=used)


def load_vcycle_counts():
    """V-cycles and smoother rebuilds per step of the timed workload, as
    measured on the GPU and committed (read only)."""
    if os.path.exists(VCYCLE_FILE):
        with open(VCYCLE_FILE) as f:
            return json.load(f)
    return None


def run_reference(args, wl, world, rank):
    if rank != 0:
        return 0
    counts = load_vcycle_counts() if args.workload == "c2" else None
    n_v, n_r = (counts["vcycles"], counts["refreshes"]) if counts else (1, 1)
    cores = os.cpu_count() or 1
    if args.warmup > 0:   # one untimed sample (page-in, first-touch), not in the median
        oracle_sample(wl, n_r, n_v - n_r, threads=cores)
    samples = [oracle_sample(wl, n_r, n_v - n_r, threads=cores) for _ in range(args.steps)]
    s = float(np.median([x["s_per_step"] for x in samples]))
    used = samples[-1]["threads"]
    E = wl["n"] ** 2
    dsw = dof_sweeps_per_vcycle(E, wl["levels"], wl["smooth"])
    sample = (f"extrapolated from sampled V-cycles: one FAS V-cycle with smoother rebuild and one without on the "
              f"full workload, FP64 oracle on {used} host threads ({cpu_model()}); scaled by {n_r} rebuilding "
              f"and {n_v - n_r} plain V-cycles per step (the GPU's committed counts)"
              + ("" if counts else " (no measured V-cycle count found: per V-cycle figure)"))
    line = {"impl": "reference", "metric": METRIC, "value": s, "unit": "s/step", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * s, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "elements": E, "parallelism": "replicas"},
            "dof_sweeps_per_s": dsw / samples[-1]["t_vcycle"],
            "cpu_baseline": {"kind": "oracle", "value": s, "unit": "s/step", "cores": used, "cpu": cpu_model(),
                             "sample": sample, "extrapolated": True},
            "e2e": {"value": s, "unit": "s/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
# Measured FP32 instructions of the double-word sweep kernels (ncu), for the
# FP32-issue roofline of those kernels; see profiles/.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz


def ncu_record():
    path = os.path.join(ROOT, "profiles", "ncu_traffic_c2.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    return rec if rec.get("csrc_sha256_prefix") == csrc_fingerprint() else None


def solution_diff(qa, qb, p_inf):
    """max |qa - qb| of the velocity and of (p - p_inf)/(rho_inf |v_inf|^2)
    (rho_inf |v_inf|^2 = 2 for the vortex)."""
    return {"u": float(np.abs(qa[1] - qb[1]).max()), "v": float(np.abs(qa[2] - qb[2]).max()),
            "p_over_rho_v2": float(np.abs(qa[0] - qb[0]).max() / 2.0),
            "T_over_T_inf": float(np.abs(qa[3] - qb[3]).max() / p_inf)}


def run_ours(args, wl, world, rank, local):
    import torch
    from paper_1908_03972_gb300 import build, pmgfr, workloads as W

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    build.build()
    pmgfr.load()
    nodes, nbr = W.periodic_box(wl["n"], wl["n"], Ng=1)
    E = nodes.shape[0]
    stream = torch.cuda.current_stream(device)
    p_inf = W.freestream_T(0.005)
    kw = dict(tol=1e-8, dtau_init=0.01, dtau_max=10.0, refresh_every=10, max_pseudo=20000, use_graph=1,
              p_gauge=p_inf, res_scale=W.freestream_scales(0.005), device_loop=args.device_loop)
    dsw = dof_sweeps_per_vcycle(E, wl["levels"], wl["smooth"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    # The three legs: (block precision, residual arithmetic of the sweeps)
    LEGS = {
        "mixed": (pmgfr.PMG_PREC_FP32, pmgfr.PMG_FLUX_DW_SMOOTH),
        "mixed_bf16": (pmgfr.PMG_PREC_BF16R, pmgfr.PMG_FLUX_DW_SMOOTH),
        "mixed_f64res": (pmgfr.PMG_PREC_FP32, pmgfr.PMG_FLUX_FP64),
        "fp64": (pmgfr.PMG_PREC_FP64, pmgfr.PMG_FLUX_FP64),
        "nk_pmg": (pmgfr.PMG_PREC_FP32, pmgfr.PMG_FLUX_DW_SMOOTH),
    }
    # Newton-Krylov stages with one V-cycle as the preconditioner (the
    # variant the paper's conclusions name as future work); the difference
    # step is taken relative to the absolute pressure and temperature scale.
    NK_OPTS = dict(precond=pmgfr.PMG_NK_PC_VCYCLE, krylov_dim=30, max_krylov=60, dtau_pc=10.0, pc_refresh=2,
                   state_scale=(p_inf, 1.0, 1.0, p_inf))

    def make(leg):
        prec, flux = LEGS[leg]
        s = pmgfr.Solver(nodes, nbr, wl["levels"], wl["smooth"], stream=stream.cuda_stream, block_prec=prec,
                         flux_prec=flux, **kw)
        if leg == "nk_pmg":
            pmgfr.pmg_set_stage_solver(s.h, pmgfr.PMG_STAGE_NK, **NK_OPTS)
        return s

    solver = make("mixed")
    q0 = W.isentropic_vortex(solver.coords())
    q0_dev = torch.from_numpy(np.ascontiguousarray(q0)).to(device)
    state_bytes = q0.nbytes

    def one_step(s, timed):
        """Advance the solver's state by one physical step (events on its stream)."""
        if timed:
            flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = pmgfr.pmg_esdirk_step(s.h, wl["dt"])
        e1.record(stream)
        torch.cuda.synchronize(device)
        return e0.elapsed_time(e1), st

    if args.ncu_window:
        # Profiling window for ncu: the stage-2 system of the first step and
        # N V-cycles of it (99.9% of a step's launches are V-cycle launches),
        # with the blocks of the mixed leg or of the BF16 leg.
        s = solver if args.ncu_blocks == "fp32" else make("mixed_bf16")
        A = 1767732205903.0 / 4055673282236.0
        odt = A * wl["dt"]
        pmgfr.pmg_set_state(s.h, 0, q0_dev)
        R = s.residual(q0)
        rho = q0[0] / q0[3]
        qc = np.stack([rho, rho * q0[1], rho * q0[2], rho * (q0[3] / 0.4 + 0.5 * (q0[1] ** 2 + q0[2] ** 2))])
        s.set_stage((qc + wl["dt"] * A * R) / odt, odt)
        s.set_state(q0)
        if args.ncu_solver == "nk":
            # one Newton-Krylov solve of the same stage system
            pmgfr.pmg_set_stage_solver(s.h, pmgfr.PMG_STAGE_NK, **NK_OPTS)
            it, drop = pmgfr.pmg_stage_solve(s.h)
            torch.cuda.synchronize(device)
            if rank == 0:
                print(json.dumps({"ncu_window": "Newton-Krylov stage", "newton": it, "drop": drop,
                                  **pmgfr.pmg_nk_stats_read(s.h)}))
        else:
            # one smoother rebuild, then plain V-cycles (a timed step has 6 rebuilds in 1930 V-cycles)
            norms = [pmgfr.pmg_vcycle(s.h, 0.01 if k == 0 else 1.0, k == 0) for k in range(args.ncu_window)]
            torch.cuda.synchronize(device)
            if rank == 0:
                print(json.dumps({"ncu_window_vcycles": args.ncu_window, "blocks": args.ncu_blocks,
                                  "first_norm": norms[0], "last_norm": norms[-1]}))
        if s is not solver:
            s.close()
        solver.close()
        return 0

    def timed_steps(s, n, sampler=None):
        if sampler:
            sampler.start()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(device)
        ms, its, drops, nvs, nrs, states = [], [], [], [], [], []
        for _ in range(n):
            t, stats = one_step(s, True)
            ms.append(t)
            its.append(list(stats.pseudo_iters)[:3])
            drops.append(max(float(x) for x in list(stats.res_drop)[:3]))
            nvs.append(stats.n_vcycles)
            nrs.append(stats.n_refresh)
            states.append(s.get_state())   # after the step's events: outside the timed step
        torch.cuda.synchronize(device)
        clocks = sampler.stop() if sampler else None
        mean_ms = barrier_max(float(np.mean(ms)), world, device)
        nv = float(np.mean(nvs))
        return dict(s_per_step=mean_ms / 1000.0, steps=n, ms=ms, vcycles=nv, refreshes=float(np.mean(nrs)),
                    pseudo_iters=its, max_res_drop=drops, dof_sweeps_per_s=dsw * nv * world / (mean_ms / 1000.0),
                    ms_per_vcycle=mean_ms / nv, clocks=clocks), states

    # Headline leg: W warm-up steps from the analytic state, then K timed
    # steps.  After the first warm-up step (which leaves stage data and a built
    # smoother) the autotuner picks each coarse level's smoothing schedule.
    pmg_tune = {}
    pmgfr.pmg_set_state(solver.h, 0, q0_dev)
    for w in range(args.warmup):
        one_step(solver, False)
        if w == 0 and not args.no_autotune:
            pmg_tune = pmgfr.pmg_autotune(solver.h, reps=3)
    q_warm = np.ascontiguousarray(solver.get_state())
    results = {}
    results["mixed"], mixed_states = timed_steps(solver, args.steps, ClockSampler(local))
    # Other legs: the same physical steps from the same warmed state (one
    # untimed step first for their own graph captures, then reset), K2 steps.
    k2 = min(args.steps, args.other_steps)
    legs = [] if args.skip_fp64 else ["mixed_bf16", "mixed_f64res", "fp64"]
    if not args.skip_nk:
        legs.append("nk_pmg")
    nk_work = {}
    diffs = {}
    for leg in legs:
        s = make(leg)
        s.set_state(q_warm)
        one_step(s, False)
        if not args.no_autotune:
            pmgfr.pmg_autotune(s.h, reps=3)
        s.set_state(q_warm)
        if leg == "nk_pmg":
            pmgfr.pmg_nk_stats_read(s.h, reset=True)
        results[leg], st = timed_steps(s, k2)
        if leg == "nk_pmg":
            nk_work = {k: v / k2 for k, v in pmgfr.pmg_nk_stats_read(s.h, reset=True).items()}
        diffs[f"mixed_vs_{leg}"] = solution_diff(mixed_states[k2 - 1], st[k2 - 1], p_inf)
        s.close()
    mixed = results["mixed"]

    # End to end through the C interface with host buffers: the same K steps
    # from the state after the warm-ups, each step taking its state from pinned
    # host memory and returning the new state there.
    qh = torch.from_numpy(q_warm).pin_memory().numpy()
    out = torch.empty(qh.shape, dtype=torch.float64).pin_memory().numpy()
    e2e = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        pmgfr.pmg_set_state(solver.h, 0, qh)
        pmgfr.pmg_esdirk_step(solver.h, wl["dt"])
        pmgfr.pmg_get_state(solver.h, 0, out)
        e2e.append(time.perf_counter() - t0)
        qh[...] = out
    e2e_s = barrier_max(float(np.mean(e2e)), world, device)

    # per-launch profile of one step (launch by launch, CUDA events on the solver stream)
    pmgfr.pmg_profile(solver.h, True)
    one_step(solver, False)
    prof = pmgfr.pmg_profile_read(solver.h)
    pmgfr.pmg_profile(solver.h, False)
    total_ms = sum(v[0] for v in prof.values())
    launches = sum(v[1] for v in prof.values())
    by_class = {}
    for (name, lvl), (t, n) in prof.items():
        by_class.setdefault(name, [0.0, 0])
        by_class[name][0] += t
        by_class[name][1] += n
    top = max(prof.items(), key=lambda kv: kv[1][0])
    (top_name, top_lvl), (top_ms, top_n) = top
    P = wl["levels"][top_lvl]
    avg_s = top_ms / top_n / 1000.0
    key = f"{top_name}[level {top_lvl}, P={P}]"
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_note = "measured" if "hbm_gbs" in peaks else "fallback"
    rec = ncu_record()
    krec = (rec or {}).get("kernels", {}).get(key, {})
    # Which pipe the dominant kernel runs on: the mixed leg's sweep kernels run
    # their arithmetic in double-word on the FP32 pipes; their roofline is FP32
    # issue, from the FP32 operations ncu counted (FFMA = 2, FADD/FMUL = 1).
    if top_name == "apply":
        work = apply_bytes(P, E, 4)
        roofline = {"bound": "hbm", "achieved": work / avg_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "peak_source": hbm_note}
    elif krec.get("fp32_flops_per_launch"):
        work = krec["fp32_flops_per_launch"]
        roofline = {"bound": "alu", "achieved": work / avg_s / 1e12, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz",
                    "work": "FP32 flops per launch counted by ncu (double-word arithmetic of the method's binary64 "
                            "operations)"}
    else:
        work = None
        roofline = {"bound": "alu", "achieved": None, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz",
                    "work": "no ncu FP32 count for the current kernel sources"}
    roofline.update({"kernel": key, "frac": (roofline["achieved"] / roofline["peak"]) if roofline["achieved"] else None,
                     "traffic": krec.get("dram_bytes_per_launch"), "share_of_step": top_ms / total_ms,
                     "avg_launch_us": avg_s * 1e6, "launches_per_step": top_n})
    # V-cycle level: the FP32 block inverses the sweeps must read per V-cycle
    # (n^2 entries per element per sweep on every level) over the V-cycle time.
    blk = sum(4 * E * (4 * (Pl + 1) ** 2) ** 2 * (n if l == len(wl["levels"]) - 1 else 2 * n)
              for l, (Pl, n) in enumerate(zip(wl["levels"], wl["smooth"])))
    vc_s = mixed["s_per_step"] / mixed["vcycles"]
    vcycle_hbm = {"block_bytes_per_vcycle": blk, "ms_per_vcycle": vc_s * 1e3, "achieved_gbs": blk / vc_s / 1e9,
                  "peak_gbs": hbm_peak, "frac": blk / vc_s / 1e9 / hbm_peak}

    # CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only), on one
    # host thread and on all of them
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        try:
            n_r, n_p = mixed["refreshes"], mixed["vcycles"] - mixed["refreshes"]
            cores = os.cpu_count() or 1
            one = oracle_sample(wl, n_r, n_p, threads=1)
            allc = oracle_sample(wl, n_r, n_p, threads=cores)
            cpu = {"value": allc["s_per_step"], "unit": "s/step", "cores": allc["threads"], "kind": "oracle",
                   "cpu": cpu_model(), "extrapolated": True, "single_core_value": one["s_per_step"],
                   "sample": ("extrapolated from sampled V-cycles: one V-cycle with smoother rebuild and one "
                              "without on the full workload, FP64 oracle, on %d host threads (%.2f s and %.2f s) "
                              "and on one (%.1f s and %.1f s), scaled by this run's %d rebuilding and %d plain "
                              "V-cycles per step" % (allc["threads"], allc["t_vcycle_refresh"], allc["t_vcycle"],
                                                     one["t_vcycle_refresh"], one["t_vcycle"], round(n_r),
                                                     round(n_p)))}
        except Exception as exc:  # the product number stands without it
            cpu = {"value": None, "unit": "s/step", "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": mixed["s_per_step"], "unit": "s/step", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mixed["s_per_step"] * 1000.0,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 residual + f32x2 (double-word) sweeps + f32 blocks",
            "data": "synthetic",
            "config": {"workload": wl["name"], "elements": E, "dofs_finest": 4 * E * (wl["levels"][0] + 1) ** 2,
                       "blocks": "FP32 equilibrated Gauss-Jordan inverse",
                       "residual": ("binary64 for the finest level's residual (stopping norm, restricted defect, "
                                    "pmg_residual); double-word (float-float, ~2^-48) in every smoothing sweep's "
                                    "residual-and-update on every level and in the coarse levels' residuals"),
                       "mixed_bf16_leg": "BF16 block inverses applied with FP32 accumulation, residuals as mixed",
                       "mixed_f64res_leg": "FP32 blocks, binary64 residual everywhere",
                       "fp64_leg": "FP64 blocks, binary64 residual everywhere",
                       "nk_pmg_leg": ("as mixed, each stage solved by Newton-Krylov (restarted FGMRES(30), "
                                      "difference Jacobian, one FAS V-cycle as the preconditioner, eta 1e-2, "
                                      "smoother rebuilt every second Newton step) "
                                      "instead of pseudo-transient continuation; pseudo_iters count Newton steps"),
                       "l2": "flushed (256 MiB write) before every timed step", "parallelism": "replicas"},
            "mixed": {k: v for k, v in mixed.items() if k not in ("clocks",)},
            "mixed_bf16": {k: v for k, v in results.get("mixed_bf16", {}).items() if k not in ("clocks",)},
            "mixed_f64res": {k: v for k, v in results.get("mixed_f64res", {}).items() if k not in ("clocks",)},
            "fp64": {k: v for k, v in results.get("fp64", {}).items() if k not in ("clocks",)},
            "nk_pmg": dict({k: v for k, v in results.get("nk_pmg", {}).items() if k not in ("clocks",)},
                           **({"per_step": nk_work} if nk_work else {})),
            "solution_diff_after_%d_steps" % k2: diffs,
            "dof_sweeps_per_vcycle": dsw,
            "autotune": {f"level {l}": v for l, v in pmg_tune.items()},
            "device_loop": args.device_loop,
            "clocks": mixed["clocks"],
            "e2e": {"value": e2e_s, "unit": "s/step", "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes},
            "gpu_launches": launches * args.steps,
            "profile_ms_by_kernel": {k: {"ms": v[0], "launches": v[1]} for k, v in sorted(by_class.items())},
            "roofline": roofline,
            "vcycle_hbm": vcycle_hbm,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0



# ------------------------------------------------------- hierarchy study
HIERARCHIES = [([4], [10]), ([4, 3], [5, 10]), ([4, 2], [5, 10]), ([4, 1], [5, 10]), ([4, 3, 2], [5, 10, 20]),
               ([4, 3, 1], [5, 10, 20]), ([4, 2, 1], [5, 10, 20])]


def run_hierarchy_study(args):
    """The P-hierarchies of the paper's P = 4 study (Section 4.2: P{4-3},
    P{4-2}, P{4-1}, P{4-3-2}, P{4-3-1}, P{4-2-1}, and the single level) on
    the cylinder workload at 1/16 of its elements (16 x 64 Q2 quads, Re = 100,
    Ma = 0.001, no-slip wall), the system of the first implicit ESDIRK3 stage
    from the free stream with 1e-3 noise in v, with gauge storage and BF16
    blocks.  Each hierarchy solves it to a 1e-8 drop twice: by the paper's
    pseudo-transient continuation (dtau 0.01 -> 1 by SER, the smoother rebuilt
    every 10 iterations throughout; dtau_max = 10 diverges, see the
    findings) and by Newton-Krylov with one V-cycle of the hierarchy as the
    preconditioner.  One JSON line per hierarchy: V-cycles and GPU seconds."""
    import torch
    from paper_1908_03972_gb300 import build, pmgfr, workloads as W
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    build.build()
    pmgfr.load()
    MA, MU = 0.001, 0.01
    T = W.freestream_T(MA, speed=1.0)
    nodes, nbr = W.cylinder_omesh(16, 64, 0.5, 50.0, Ng=2)
    stream = torch.cuda.current_stream()
    for levels, smooth in HIERARCHIES:
        out = {"study": "hierarchy", "workload": "cylinder 16x64 Q2 quads (1/16 of 64x256), Re 100, Ma 0.001, "
                                                 "first implicit ESDIRK3 stage (dt 0.05) from the free stream",
               "hierarchy": "P{" + "-".join(map(str, levels)) + "}", "smoothing": "I{" + "-".join(map(str, smooth)) + "}"}
        for solver in ("ptc", "nk"):
            s = pmgfr.Solver(nodes, nbr, levels, smooth, stream=stream.cuda_stream, block_prec=pmgfr.PMG_PREC_BF16R,
                             Ma_inf=MA, mu=MU, cutoff=1, kappa=1.0, q_inf=(T, 1.0, 0.0, T), p_gauge=T,
                             res_scale=W.freestream_scales(MA, speed=1.0), tol=1e-8, dtau_init=0.01, dtau_max=1.0,
                             refresh_every=10, refresh_always=1, max_pseudo=20000)
            try:
                if solver == "nk":
                    pmgfr.pmg_set_stage_solver(s.h, pmgfr.PMG_STAGE_NK, precond=pmgfr.PMG_NK_PC_VCYCLE,
                                               krylov_dim=30, max_krylov=60, dtau_pc=1.0, max_newton=40,
                                               state_scale=(T, 1.0, 1.0, T))
                q = W.freestream_noise_state(s.coords(), MA)
                rho = q[0] / q[3]
                qc = np.stack([rho, rho * q[1], rho * q[2], rho * (q[3] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2))])
                A = 1767732205903.0 / 4055673282236.0
                odt = A * 0.05
                s.set_stage((qc + 0.05 * A * s.residual(q)) / odt, odt)
                s.set_state(q)
                pmgfr.pmg_nk_stats_read(s.h, reset=True)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                try:
                    it, drop = pmgfr.pmg_stage_solve(s.h)
                    status = "converged"
                except pmgfr.PmgError as ex:
                    it, drop, status = -1, float("nan"), str(ex)
                torch.cuda.synchronize()
                sec = time.perf_counter() - t0
                rec = {"status": status, "seconds": sec, "drop": drop}
                if solver == "nk":
                    st = pmgfr.pmg_nk_stats_read(s.h)
                    rec.update(newton=it, vcycles=st["vcycles"], residuals=st["residuals"])
                else:
                    rec.update(vcycles=it)
                out[solver] = rec
            finally:
                s.close()
        print(json.dumps(out), flush=True)
    return 0


def run_cylinder_study(args):
    """The cylinder workload (Re = 100, Ma = 0.001, no-slip wall, P{4-2-1},
    I{5-10-20}, ESDIRK3 dt = 0.05, from the free stream with 1e-3 noise in v,
    gauge storage) with Newton-Krylov stages and one V-cycle as the
    preconditioner (its pseudo-transient solve diverges, see the findings),
    BF16, FP32 and FP64 blocks: consecutive steps of the mesh at 1/16 of its
    elements (16 x 64) and at full size (64 x 256).  One JSON line per
    (mesh, blocks): seconds, Newton steps, V-cycles and status of each step."""
    import torch
    from paper_1908_03972_gb300 import build, pmgfr, workloads as W
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    build.build()
    pmgfr.load()
    MA, MU = 0.001, 0.01
    T = W.freestream_T(MA, speed=1.0)
    stream = torch.cuda.current_stream()
    for (nr, nt, nsteps) in ((16, 64, 3), (64, 256, 2)):
        nodes, nbr = W.cylinder_omesh(nr, nt, 0.5, 50.0, Ng=2)
        for prec, name in ((pmgfr.PMG_PREC_BF16R, "bf16"), (pmgfr.PMG_PREC_FP32, "fp32"),
                           (pmgfr.PMG_PREC_FP64, "fp64")):
            s = pmgfr.Solver(nodes, nbr, [4, 2, 1], [5, 10, 20], stream=stream.cuda_stream, block_prec=prec,
                             Ma_inf=MA, mu=MU, cutoff=1, kappa=1.0, q_inf=(T, 1.0, 0.0, T), p_gauge=T,
                             res_scale=W.freestream_scales(MA, speed=1.0), tol=1e-8, dtau_max=10.0)
            steps = []
            try:
                pmgfr.pmg_set_stage_solver(s.h, pmgfr.PMG_STAGE_NK, precond=pmgfr.PMG_NK_PC_VCYCLE, krylov_dim=50,
                                           max_krylov=200, dtau_pc=0.1, max_newton=60, state_scale=(T, 1.0, 1.0, T))
                s.set_state(W.freestream_noise_state(s.coords(), MA))
                for k in range(nsteps):
                    pmgfr.pmg_nk_stats_read(s.h, reset=True)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    status, st = pmgfr.pmg_esdirk_step(s.h, 0.05, raise_on_error=False)
                    torch.cuda.synchronize()
                    sec = time.perf_counter() - t0
                    ks = pmgfr.pmg_nk_stats_read(s.h, reset=True)
                    steps.append({"seconds": sec, "status": "converged" if status == 0 else pmgfr.pmg_last_error(),
                                  "newton": list(st.pseudo_iters[:3]), "drops": list(st.res_drop[:3]),
                                  "vcycles": ks["vcycles"], "residuals": ks["residuals"]})
                    if status:
                        break
            finally:
                s.close()
            print(json.dumps({"study": "cylinder", "mesh": f"{nr}x{nt}", "elements": nr * nt, "blocks": name,
                              "stage_solver": "Newton-Krylov, FGMRES(50), one V-cycle preconditioner, dtau_pc 0.1",
                              "steps": steps}), flush=True)
    return 0

def run_ellipse_study(args):
    """The extruded-ellipse workload (chord 1, thickness 0.1, incidence 8
    degrees, O-mesh 48 radial x 64 around x 20 spanwise hexahedra over a span
    of 0.2, periodic in z, far field at 20 chords; P{3-2-1-0}, I{5-10-20-40},
    Re = 60000, Ma = 0.1 and 0.01, no-slip wall, gauge storage), FP32 and
    FP64 blocks: the time of a residual, of the smoother's rebuild (assembly
    and factorisation of every level's blocks) and of a V-cycle, and the
    first ESDIRK3 step (dt = 0.001) from the free stream with 1e-3 noise in v
    by Newton-Krylov stages with one V-cycle as the preconditioner (dtau_pc
    1e-3, blocks rebuilt every second Newton step; at dt = 0.01 the
    preconditioner's V-cycle returns non-finite directions in the first
    stage).  One JSON line per (Ma, blocks); the step with FP32 blocks only."""
    import torch
    from paper_1908_03972_gb300 import build, pmgfr, workloads as W
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    build.build()
    pmgfr.load()
    nr, nt, nz = {"full": (48, 64, 20), "half": (24, 32, 10), "small": (12, 16, 5)}[args.study_mesh]
    nodes, nbr = W.extruded_ellipse(nr, nt, nz, span=0.2, Ng=2)
    alpha = math.radians(8.0)
    stream = torch.cuda.current_stream()
    if args.ncu_window > 0:   # profiling helper: one V-cycle with rebuild, then N without (Ma = 0.1, FP32)
        MA = 0.1
        T = W.freestream_T(MA, speed=1.0)
        qinf = (T, math.cos(alpha), math.sin(alpha), 0.0, T)
        s = pmgfr.Solver(nodes, nbr, [3, 2, 1, 0], [5, 10, 20, 40], stream=stream.cuda_stream,
                         block_prec=pmgfr.PMG_PREC_FP32, dim=3, Ma_inf=MA, mu=1.0 / 60000.0, cutoff=1, kappa=1.0,
                         q_inf3=qinf, p_gauge=T, res_scale3=W.freestream_scales3(MA, speed=1.0))
        try:
            xyz = s.coords()
            q = W.uniform_state3(xyz.shape[0], xyz.shape[1], T, qinf[1], qinf[2], 0.0, T)
            q[2] += 1e-3 * np.random.default_rng(7).standard_normal(q.shape[1:])
            rho = q[0] / q[4]
            qc = np.stack([rho, rho * q[1], rho * q[2], rho * q[3],
                           rho * (q[4] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2))])
            s.set_stage(qc / 0.005, 0.005)
            s.set_state(q)
            norms = [pmgfr.pmg_vcycle(s.h, 1e-3, True)]
            norms += [pmgfr.pmg_vcycle(s.h, 1e-3, False) for _ in range(args.ncu_window)]
            torch.cuda.synchronize()
            print(json.dumps({"ncu_window_vcycles": args.ncu_window + 1, "workload": "extruded ellipse",
                              "first_norm": norms[0], "last_norm": norms[-1]}))
        finally:
            s.close()
        return 0
    for MA in (0.1, 0.01):
        T = W.freestream_T(MA, speed=1.0)
        qinf = (T, math.cos(alpha), math.sin(alpha), 0.0, T)
        precs = ((pmgfr.PMG_PREC_FP32, "fp32"), (pmgfr.PMG_PREC_FP64, "fp64"))
        for prec, name in precs[:1] if args.study_fp32_only else precs:
            rec = {"study": "ellipse", "mesh": f"{nr}x{nt}x{nz}", "elements": nr * nt * nz, "Ma": MA,
                   "Re": 60000, "blocks": name, "levels": "P{3-2-1-0}, I{5-10-20-40}"}
            s = pmgfr.Solver(nodes, nbr, [3, 2, 1, 0], [5, 10, 20, 40], stream=stream.cuda_stream, block_prec=prec,
                             dim=3, Ma_inf=MA, mu=1.0 / 60000.0, cutoff=1, kappa=1.0, q_inf3=qinf, p_gauge=T,
                             res_scale3=W.freestream_scales3(MA, speed=1.0), tol=1e-8, dtau_max=1.0)
            try:
                xyz = s.coords()
                E, N = xyz.shape[0], xyz.shape[1]
                q = W.uniform_state3(E, N, T, qinf[1], qinf[2], 0.0, T)
                q[2] += 1e-3 * np.random.default_rng(7).standard_normal((E, N))
                s.set_state(q)

                def timed(fn, reps):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    for _ in range(reps):
                        fn()
                    torch.cuda.synchronize()
                    return (time.perf_counter() - t0) / reps

                dev = torch.device("cuda", torch.cuda.current_device())
                q_dev = torch.from_numpy(np.ascontiguousarray(q)).to(dev)
                r_dev = torch.empty_like(q_dev)
                rec["residual_s"] = timed(lambda: pmgfr.pmg_residual(s.h, 0, q_dev, r_dev), 3)
                del q_dev, r_dev
                # a stage system of the size of an implicit stage with omega dt = 0.005
                rho = q[0] / q[4]
                qc = np.stack([rho, rho * q[1], rho * q[2], rho * q[3],
                               rho * (q[4] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2))])
                odt = 0.005
                s.set_stage(qc / odt, odt)
                rec["vcycle_rebuild_s"] = timed(lambda: pmgfr.pmg_vcycle(s.h, 1e-3, True), 2)
                rec["vcycle_s"] = timed(lambda: pmgfr.pmg_vcycle(s.h, 1e-3, False), 5)
                rec["rebuild_s"] = rec["vcycle_rebuild_s"] - rec["vcycle_s"]
                if name == "fp32":   # the first step with FP32 blocks only
                    pmgfr.pmg_set_stage_solver(s.h, pmgfr.PMG_STAGE_NK, precond=pmgfr.PMG_NK_PC_VCYCLE,
                                               krylov_dim=30, max_krylov=40, dtau_pc=1e-3, max_newton=10,
                                               pc_refresh=args.nk_pc_refresh, state_scale=(T, 1.0, 1.0, 1.0, T))
                    s.set_state(q)
                    pmgfr.pmg_nk_stats_read(s.h, reset=True)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    status, st = pmgfr.pmg_esdirk_step(s.h, 0.001, raise_on_error=False)
                    torch.cuda.synchronize()
                    ks = pmgfr.pmg_nk_stats_read(s.h, reset=True)
                    rec["first_step"] = {"dt": 0.001, "pc_refresh": args.nk_pc_refresh,
                                         "seconds": time.perf_counter() - t0,
                                         "status": "converged" if status == 0 else pmgfr.pmg_last_error(),
                                         "newton": list(st.pseudo_iters[:3]), "drops": list(st.res_drop[:3]),
                                         "vcycles": ks["vcycles"]}
            except Exception as exc:   # report what was measured before the failure
                rec["error"] = str(exc)
            finally:
                s.close()
            print(json.dumps(rec), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--skip-fp64", action="store_true", help="skip the BF16, binary64-residual and FP64 legs")
    ap.add_argument("--skip-nk", action="store_true", help="skip the Newton-Krylov leg")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default coarse-level schedule")
    ap.add_argument("--device-loop", type=int, default=0, choices=[0, 1],
                    help="1: each stage's pseudo-iterations as one CUDA graph with a conditional WHILE node")
    ap.add_argument("--other-steps", type=int, default=4,
                    help="timed steps of the mixed_f64res and fp64 legs (at most --steps)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--ncu-window", type=int, default=0,
                    help="profiling helper: run N V-cycles of the first stage and exit (no bench line)")
    ap.add_argument("--ncu-blocks", default="fp32", choices=["fp32", "bf16"],
                    help="block precision of the --ncu-window run")
    ap.add_argument("--ncu-solver", default="ptc", choices=["ptc", "nk"],
                    help="nk: the --ncu-window run is one Newton-Krylov solve of the stage instead of N V-cycles")
    ap.add_argument("--study", default="", choices=["", "hierarchy", "cylinder", "ellipse"],
                    help="hierarchy: the P-hierarchy study on the reduced cylinder; cylinder: Newton-Krylov steps of "
                         "the cylinder workload; ellipse: the extruded-ellipse workload's residual, rebuild, "
                         "V-cycle and first stage (JSON lines, no bench line)")
    ap.add_argument("--study-fp32-only", action="store_true", help="the ellipse study without its FP64 legs")
    ap.add_argument("--nk-pc-refresh", type=int, default=2,
                    help="the ellipse study's step: rebuild the preconditioner's blocks every N Newton steps")
    ap.add_argument("--study-mesh", default="full", choices=["full", "half", "small"],
                    help="the ellipse study's mesh: 48 x 64 x 20, 24 x 32 x 10 or 12 x 16 x 5 elements")
    args = ap.parse_args()
    if args.study == "hierarchy":
        return run_hierarchy_study(args)
    if args.study == "cylinder":
        return run_cylinder_study(args)
    if args.study == "ellipse":
        return run_ellipse_study(args)
    world, rank, local = dist_setup()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl, world, rank)
    return run_ours(args, wl, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
