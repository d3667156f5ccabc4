#!/usr/bin/env python3
"""Benchmark: converged state-steps/s of the parallel-Newton solve on the batched
mass-action workload (B = 4096 random networks, d = 8, 12 reactions, RK4 dt = 1e-3,
T = 16384, full-Jacobian Newton, FP32 with a compensated state, converged when
max |r| / max(1, |s|) <= 5e-8 on two consecutive iterates, zero initial guess, reset
heuristic on, sliding window).

One step = one deer_solve of the whole batch to convergence (every Newton iteration:
linearise + residual, convergence check, parallel scan), inputs resident in HBM.
Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle instead.

Multi-GPU (torchrun): every rank solves its own 4096 trajectories (independent problems,
no data-path collective; weak scaling); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# window: the sliding window of Sec. 3.2 (converged prefixes are frozen), which the thesis
# recommends for every parallel Newton solve
# tol: scaled residual 5e-8 on two consecutive iterates, which the compensated float32
# state (a float32 low-order term per state entry) can meet: its residual is accurate to
# the rounding of the integrator increments, not to a float32 ulp of the state
# initial guess: the constant s_0 (6 % faster than zeros on this workload: Newton
# iterations p50 6 / max 60 against 7 / 80; the fixed point is the same)
WORKLOAD = dict(B=4096, d=8, R=12, T=16384, dt=1e-3, integrator="rk4", tol=5e-8,
                confirm=2, init="s0", window=True)
METRIC = "converged state-steps/sec vs sequential rollout; scan GB/s or TC % of peak"
UNIT = "state-steps/s"
CONFIG_NAME = ("batched mass-action networks B=4096 d=8 R=12 RK4 dt=1e-3 T=16384, "
               "full-Jacobian Newton, FP32")
# Algorithmic work per trajectory row of one Newton iteration of the headline workload
# (d = 8, RK4), as the measurement plan fixes it: the step Jacobian by the chain rule through
# the stages (3 products of 8x8 matrices, 3 * 2 d^3 = 3072 flop), the composition of the
# affine scan element (2 d^3 + 2 d^2 = 1152 flop) and four rate evaluations (~300 flop):
# 4524 flop; and, with A_t kept on chip, s_{t-1} and s_t read and s written: 3 * d * 4 = 96 B.
ALGO_FLOP_PER_ROW = 3 * 2 * 8 ** 3 + (2 * 8 ** 3 + 2 * 8 ** 2) + 300
ALGO_BYTES_PER_ROW = 3 * 8 * 4
# What the fused kernel moves per row by design: the pending Jacobian and offset of the
# previous iteration read and the new ones written (d^2 + d each way), the state and its
# float32 compensation term read and written.
IMPL_BYTES_PER_ROW = 2 * (8 * 8 + 8) * 4 + 2 * 2 * 8 * 4
# DRAM bytes per row of the fused iteration kernel from the committed ncu capture of the
# same kernel (dram__bytes_read.sum + dram__bytes_write.sum per row at B=512, two launches:
# 4.407 GB / 6.29 M rows and 2.517 GB / 3.62 M rows; the traffic per row does not depend on
# B), scaled by the rows of an average launch; None while the kernel has changed since its
# capture.
FUSED_TRAFFIC_PER_ROW = (4.407065e9 + 2.516884e9) / (6285312 + 3622912)
# Mixed-precision d=16 mass-action linearise, per row: the RK4 step Jacobian chain in
# float32 (3 products of 16x16 matrices, 3 * 2 d^3 flop); the float64 rate evaluations are
# not counted.
MIXED_LIN_FLOP_PER_ROW = 3 * 2 * 16 ** 3


def _rel_err_per_seq(got, ref, off):
    """Normwise error of every sequence of a packed batch: max |got - ref| / max |ref|."""
    import numpy as np
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    out = np.zeros(len(off) - 1)
    for b in range(len(off) - 1):
        lo, hi = int(off[b]), int(off[b + 1])
        if hi > lo:
            out[b] = np.max(np.abs(got[lo:hi] - ref[lo:hi])) / max(np.max(np.abs(ref[lo:hi])),
                                                                    1e-300)
    return out


class OracleChecks:
    """Comparisons of GPU results with the FP64 oracle. Each measurement registers a
    closure over host copies of its results; they all run in the CPU-baseline leg, after
    every GPU timing, and fill each entry's ``max_rel_err_vs_oracle``."""

    def __init__(self):
        self.items = []

    def add(self, entry: dict, fn):
        self.items.append((entry, fn))

    def run(self):
        for entry, fn in self.items:
            t0 = time.perf_counter()
            res = fn()
            entry.update(res)
            entry["oracle_check_s"] = round(time.perf_counter() - t0, 2)


def _peaks():
    """HBM copy bandwidth and cuBLAS bf16 rate of this GPU model, with where they came
    from: the measured MEASURED_PEAKS.json when present, else one earlier GB300
    measurement (6.8 TB/s copy, 1.9 PFLOP/s bf16), reported as the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured (MEASURED_PEAKS.json)"
    return ({"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0},
            "fallback (no MEASURED_PEAKS.json: an earlier GB300 measurement)")


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    def __init__(self, index: int, path: str):
        self.path, self.proc = path, None
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(value: float, device=None) -> float:
    """Largest value over the ranks of the job (identity on one rank): the step time every
    rank reports is the slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _whole_job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Throughput of the whole job: every rank solves its own batch (replicas, weak
    scaling) in at most `ms` (the max over ranks)."""
    return world * units_per_rank / (ms / 1000.0)


def _problem(rank: int, batch: int = 0):
    import synth
    w = WORKLOAD
    return synth.massaction(batch or w["B"], w["d"], w["R"], w["T"], seed=rank, dt=w["dt"],
                            integrator=w["integrator"])


def cpu_oracle_rollout(p, threads=None):
    """The FP64 oracle's answer for the headline workload, timed: the sequential rollout
    s_t = f(s_{t-1}) of every trajectory in plain C (oracle/c/massaction.c), the batch split
    over `threads` host threads (default: every core). Returns (rollout [B*T][d], seconds,
    threads used)."""
    from oracle import cma
    B, T = p["topology"].shape[0], p["T"]
    threads = threads or cma.cores()
    batch = cma.Batch(p["topology"], p["params"], p["dt"], "rk4", d=p["d"])
    off = cma.uniform_offsets(B, T)
    t0 = time.perf_counter()
    ref = batch.rollout(p["s0"], off, threads=threads)
    return ref, time.perf_counter() - t0, threads


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    p = _problem(0)
    B, T = WORKLOAD["B"], WORKLOAD["T"]
    for _ in range(args.warmup):
        cpu_oracle_rollout(p)
    times = []
    threads = 1
    for _ in range(args.steps):
        _, dt, threads = cpu_oracle_rollout(p)
        times.append(dt)
    total = sum(times)
    value = B * T * len(times) / total
    sample = (f"the whole workload per step: all {B} trajectories x {T} steps, FP64 oracle "
              f"sequential rollout in plain C on {threads} host threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": CONFIG_NAME, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _gru_oracle_check(g, s_host, pick, cache):
    """Normwise error of the picked GRU trajectories against the FP64 oracle rollout (the
    rollout is computed once per problem and shared by the quasi-DEER and quasi-ELK
    entries)."""
    import numpy as np
    from oracle import dynamics as odyn
    from oracle import newton as onewton
    key = tuple(int(b) for b in pick)
    if key not in cache:
        sub = odyn.GRU(g["W"], g["U"], g["x"][list(key)].astype(np.float64))
        cache[key] = onewton.rollout(sub, g["s0"][list(key)], g["x"].shape[1])
    ref = cache[key]
    T, d = ref.shape[1], ref.shape[2]
    off = [i * T for i in range(len(key) + 1)]
    err = _rel_err_per_seq(s_host.reshape(-1, d), ref.reshape(-1, d), off)
    return {"max_rel_err_vs_oracle": float(err.max()),
            "oracle_sample": f"{len(key)} of {g['x'].shape[0]} trajectories, FP64 numpy rollout"}


def gru_diag_measurement(deer, N, lib, dev, stream, steps=3, B=64, window=False, checks=None,
                         gru_cache=None):
    """GRU cell d=64, inputs 64, T=65536, B=64, weights N(0,1/d), inputs N(0,1), quasi-DEER
    (diagonal Jacobian), FP32: converged state-steps/s and the single-pass look-back
    diagonal scan in achieved HBM GB/s (algorithmic 12 bytes per coordinate-step: a, b read,
    s written)."""
    import numpy as np
    import torch
    import synth
    T, d = 65536, 64
    g = synth.gru(B, T, d, d, seed=0, dtype=np.float32)
    dyn = deer.Dynamics.gru(torch.tensor(g["W"], dtype=torch.float32, device=dev),
                            torch.tensor(g["U"], dtype=torch.float32, device=dev))
    x = torch.tensor(g["x"].reshape(-1, d), device=dev)
    s0 = torch.zeros((B, d), dtype=torch.float32, device=dev)
    opts = dict(jac="diag", tol=1e-5, confirm=2, prec="fp32", init="zeros", window=window)
    nbytes = deer.deer_workspace_bytes(dyn, B, B * T, **opts)
    ws_ = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    for _ in range(2):
        deer.deer_solve(dyn, s0, T, x, workspace=ws_, stream=stream, **opts)
    torch.cuda.synchronize()
    lib.deer_profile_reset()
    lib.deer_profile_enable(1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        s, info = deer.deer_solve(dyn, s0, T, x, workspace=ws_, stream=stream, **opts)
    e1.record(stream)
    torch.cuda.synchronize()
    lib.deer_profile_enable(0)
    prof = N.deer_profile()
    lib.deer_profile_read(prof)
    ms = e0.elapsed_time(e1) / steps
    scan_ms = prof.ms[3] / max(prof.launches[3], 1)
    scan_rows = prof.rows[3] / max(prof.launches[3], 1)
    lin_ms = prof.ms[1] / max(prof.launches[1], 1)
    lin_rows = prof.rows[1] / max(prof.launches[1], 1)
    peaks, peak_kind = _peaks()
    gbs = scan_rows * d * 12 / (scan_ms / 1000.0) / 1e9
    lin_tf = lin_rows * 4 * 2 * d * d / (lin_ms / 1000.0) / 1e12
    if int(lib.deer_get_tensor_cores()):
        # three products per row on tcgen05 kind::tf32, each as three split MMAs: the
        # tensor pipe executes 3x the useful flops
        tf32_peak, tf32_src = _tf32_peak(lib, peaks)
        lin_entry = {"kernel": "k_gru_lin_tc (tcgen05 kind::tf32, 3-term split)",
                     "avg_launch_ms": lin_ms, "achieved_tflops": lin_tf,
                     "flop_per_row": 4 * 2 * d * d,
                     "tensor_pipe_tflops": 3 * lin_tf, "tf32_peak_tflops": tf32_peak,
                     "tf32_peak_source": tf32_src, "tensor_frac": 3 * lin_tf / tf32_peak}
    else:
        lin_entry = {"kernel": "k_gru_lin_tiled", "avg_launch_ms": lin_ms,
                     "achieved_tflops": lin_tf, "flop_per_row": 4 * 2 * d * d}
    out = {"workload": f"GRU d=64 d_in=64 T=65536 B={B}, quasi-DEER, FP32, tol 1e-5 x2",
           "value": B * T / (ms / 1000.0), "unit": UNIT, "ms_per_solve": ms,
           "newton_iters_max": int(info.iters.max()), "converged": bool(info.converged.all()),
           "diag_scan": {"kernel": "k_diag_lb<float,64>", "bound": "hbm", "achieved": gbs,
                         "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / peaks["hbm_gbs"], "peak_source": peak_kind,
                         "avg_launch_ms": scan_ms,
                         "avg_rows_per_launch": scan_rows},
           "linearize": lin_entry}
    if checks is not None:
        pick = sorted(set(range(7)) | {int(info.iters.argmax())})
        s_host = s.view(B, T, d)[torch.as_tensor(pick, device=dev)].cpu().numpy()
        cache = gru_cache if gru_cache is not None else {}
        checks.add(out, lambda: _gru_oracle_check(g, s_host, pick, cache))
    return out

def brusselator_measurement(deer, dev, stream, reps=20, checks=None, N=None, lib=None):
    """C1: one Brusselator trajectory (d=2, a=1, b=3, s0=(1,1), explicit Euler dt=0.01,
    T=1024), full-Jacobian Newton in FP64 to tol 1e-12 (reset heuristic on: undamped Newton
    from the constant guess overflows on this limit cycle). The library runs a sequence this
    short whole in one kernel (a thread-block cluster iterates it to convergence); reported
    as time per solve through the API (host work included) and the kernel's own time from
    the library's phase events, next to the multi-kernel loop and the sequential GPU
    rollout."""
    import torch
    import synth
    p = synth.brusselator(T=1024)
    dyn = deer.Dynamics.brusselator(torch.tensor(p["params"], device=dev), p["dt"])
    s0 = torch.tensor(p["s0"], device=dev)
    opts = dict(jac="full", tol=1e-12, prec="fp64", init="s0", reset=True)
    ws_ = torch.empty(deer.deer_workspace_bytes(dyn, 1, 1024, **opts), dtype=torch.uint8,
                      device=dev)

    def per_call(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        e0.record(stream)
        for _ in range(reps):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    ms, (s, info) = per_call(
        lambda: deer.deer_solve(dyn, s0, 1024, workspace=ws_, stream=stream, **opts))
    kernel_us = None
    if lib is not None and N is not None:
        lib.deer_profile_reset()
        lib.deer_profile_enable(1)
        for _ in range(reps):
            deer.deer_solve(dyn, s0, 1024, workspace=ws_, stream=stream, **opts)
        torch.cuda.synchronize()
        lib.deer_profile_enable(0)
        prof = N.deer_profile()
        lib.deer_profile_read(prof)
        kernel_us = 1000.0 * sum(prof.ms) / reps
    # the multi-kernel loop on the same problem, its chunk length from the autotuner
    from paper_2603_16850_gb300 import autotune
    mopts = dict(opts, block_solve=False)
    tuned = autotune.pick_best(
        (8, 16, 32, 64, 128),
        lambda L: _time_solve1(deer, dyn, s0, 1024, None, dict(mopts, chunk=L), stream))
    mopts["chunk"] = tuned["chunk"]
    multi_ms, _ = per_call(
        lambda: deer.deer_solve(dyn, s0, 1024, workspace=ws_, stream=stream, **mopts))
    roll_ms, _ = per_call(lambda: deer.deer_rollout(dyn, s0, 1024, prec="fp64", stream=stream))
    it = int(info.iters[0])
    out = {"workload": "Brusselator d=2 T=1024 Euler dt=0.01, full Newton FP64, tol 1e-12",
           "us_per_solve": 1000 * ms, "newton_iters": it,
           "us_per_iteration": 1000 * ms / max(it, 1), "converged": bool(info.converged[0]),
           "value": 1024 / (ms / 1000.0), "unit": UNIT,
           "path": "whole solve in one kernel (one thread-block cluster)",
           "kernel_us": kernel_us,
           "multi_kernel_loop_us_per_solve": 1000 * multi_ms,
           "multi_kernel_loop_chunk": tuned["chunk"],
           "sequential_gpu_rollout_us": 1000 * roll_ms}
    if checks is not None:
        s_host = s.cpu().numpy()

        def check():
            from oracle import dynamics as odyn
            from oracle import newton as onewton
            ref = onewton.rollout(odyn.Brusselator(p["params"], p["dt"]), p["s0"], 1024)[0]
            err = _rel_err_per_seq(s_host, ref, [0, 1024])
            return {"max_rel_err_vs_oracle": float(err.max()),
                    "oracle_sample": "the whole trajectory, FP64 numpy rollout"}
        checks.add(out, check)
    return out

def gru_elk_measurement(deer, dev, stream, B=64, lams=(0.01, 0.1, 1.0, 10.0), checks=None,
                        gru_cache=None):
    """The damped variant of the GRU workload (quasi-ELK, Sec. 4.3 with the diagonal
    Jacobian): the same d=64, T=65536, B=64 problem, FP32, tol 1e-5 x2, for a sweep of the
    damping lambda = 1/sigma^2 (lambda -> 0 is quasi-DEER; larger lambda damps more, and
    the untrained GRU is contracting, so damping only slows it down: lambda = 100 and 1000
    did not converge within 2000 iterations). Converged state-steps/s and Newton
    iterations per lambda."""
    import numpy as np
    import torch
    import synth
    T, d = 65536, 64
    g = synth.gru(B, T, d, d, seed=0, dtype=np.float32)
    dyn = deer.Dynamics.gru(torch.tensor(g["W"], dtype=torch.float32, device=dev),
                            torch.tensor(g["U"], dtype=torch.float32, device=dev))
    x = torch.tensor(g["x"].reshape(-1, d), device=dev)
    s0 = torch.zeros((B, d), dtype=torch.float32, device=dev)
    rows = []
    pick = list(range(8))
    cache = gru_cache if gru_cache is not None else {}
    for lam in lams:
        opts = dict(jac="diag", damp="elk", damp_param=lam, tol=1e-5, confirm=2, prec="fp32",
                    init="zeros", max_iters=1000)
        ws_ = torch.empty(deer.deer_workspace_bytes(dyn, B, B * T, **opts), dtype=torch.uint8,
                          device=dev)
        deer.deer_solve(dyn, s0, T, x, workspace=ws_, stream=stream, **opts)  # warm
        torch.cuda.synchronize()
        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        e0.record(stream)
        s, info = deer.deer_solve(dyn, s0, T, x, workspace=ws_, stream=stream, **opts)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        row = {"lambda": lam, "value": B * T / (ms / 1000.0), "unit": UNIT, "ms": ms,
               "newton_iters_max": int(info.iters.max()),
               "converged": bool(info.converged.all())}
        rows.append(row)
        if checks is not None:
            s_host = s.view(B, T, d)[:len(pick)].cpu().numpy()
            checks.add(row, lambda s_host=s_host: _gru_oracle_check(g, s_host, pick, cache))
        del ws_
    return {"workload": f"GRU d=64 d_in=64 T=65536 B={B}, quasi-ELK (diagonal Kalman-filter "
                        "step), FP32, tol 1e-5 x2", "sweep": rows}

def lle_measurement(deer, dyn, s0, s, T, d, stream, n_sys=64):
    """Largest Lyapunov exponent (Ch. 5) along the converged trajectories of the first
    n_sys systems of the headline workload: the thesis's predictor of parallel-Newton
    convergence (negative: predictable, fast; positive: chaotic, slow)."""
    import torch
    sub = deer.Dynamics.massaction(dyn.topology[:n_sys].contiguous(),
                                   dyn.params[:n_sys].contiguous(), d, dyn.dt)
    u0 = torch.full((n_sys, d), d ** -0.5, dtype=s.dtype, device=s.device)
    traj = s.view(-1, T, d)[:n_sys].reshape(-1, d)
    torch.cuda.synchronize()
    e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    e0.record(stream)
    lle = deer.deer_lle(sub, s0[:n_sys].contiguous(), T, traj, u0, prec="fp32", stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    v = lle.cpu().numpy()
    return {"what": f"LLE estimate along the converged trajectories of {n_sys} systems",
            "min": float(v.min()), "median": float(sorted(v)[len(v) // 2]),
            "max": float(v.max()), "ms": e0.elapsed_time(e1)}


def adjoint_measurement(deer, N, lib, dev, stream, checks=None, B=256):
    """Differentiation workload: d=32 kinetic networks (48 reactions), B=256, T=32768, RK4
    dt=1e-3, FP32. Forward full-Jacobian solve, then the adjoint gradient of
    sum_t ||s_t - y_t||^2 w.r.t. the rate constants (targets y: the sequential rollout with
    rate constants k exp(0.1 eps); the timed gradient takes them from the GPU rollout, the
    oracle check from the FP64 oracle's)."""
    import numpy as np
    import torch
    import synth
    d, R, T = 32, 48, 32768
    p = synth.massaction(B, d, R, T, seed=3)
    topo = torch.tensor(p["topology"], dtype=torch.int32, device=dev)
    k = torch.tensor(p["params"], dtype=torch.float32, device=dev)
    kp_np = synth.perturbed_rates(p["params"], seed=4)
    kp = torch.tensor(kp_np, dtype=torch.float32, device=dev)
    s0 = torch.tensor(p["s0"], dtype=torch.float32, device=dev)
    dyn = deer.Dynamics.massaction(topo, k, d, p["dt"])
    y = deer.deer_rollout(deer.Dynamics.massaction(topo, kp, d, p["dt"]), s0, T, prec="fp32")
    opts = dict(jac="full", tol=5e-8, confirm=2, prec="fp32", init="zeros", reset=True)
    ws_ = torch.empty(deer.deer_workspace_bytes(dyn, B, B * T, **opts), dtype=torch.uint8,
                      device=dev)
    s, info = deer.deer_solve(dyn, s0, T, workspace=ws_, stream=stream, **opts)  # warm
    g = 2.0 * (s - y)
    gws = torch.empty(int(N.load().deer_grad_workspace_bytes(
        C.byref(dyn.c_struct()), B, T, C.byref(deer._options(**deer._opt_defaults(
            dict(prec="fp32")))))), dtype=torch.uint8, device=dev)
    deer.deer_grad(dyn, s0, T, s, g, prec="fp32", workspace=gws, stream=stream)  # warm
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    s, info = deer.deer_solve(dyn, s0, T, workspace=ws_, stream=stream, **opts)
    e1.record(stream)
    g = 2.0 * (s - y)
    dk, ds0 = deer.deer_grad(dyn, s0, T, s, g, prec="fp32", workspace=gws, stream=stream)
    e2.record(stream)
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1)
    grad = e1.elapsed_time(e2)
    # one more forward solve with the library's per-phase events (not the timed one)
    lib.deer_profile_reset()
    lib.deer_profile_enable(1)
    deer.deer_solve(dyn, s0, T, workspace=ws_, stream=stream, **opts)
    torch.cuda.synchronize()
    lib.deer_profile_enable(0)
    prof = N.deer_profile()
    lib.deer_profile_read(prof)
    del ws_
    e0.record(stream)
    deer.deer_rollout(dyn, s0, T, prec="fp32", stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    roll_ms = e0.elapsed_time(e1)
    out = {"workload": f"mass action d=32 R=48 B={B} T=32768 RK4, FP32 (compensated state, "
                       "tol 5e-8 x2), adjoint wrt rates",
           "sequential_gpu_rollout": {"ms": roll_ms, "value": B * T / (roll_ms / 1000.0),
                                      "unit": UNIT},
           "forward_ms": fwd, "grad_ms": grad,
           "forward_phase_ms": {n: prof.ms[i] for i, n in enumerate(N.PHASES)},
           "forward_rows_linearized": int(prof.rows[1]),
           "forward_value": B * T / (fwd / 1000.0), "grad_value": B * T / (grad / 1000.0),
           "unit": UNIT, "newton_iters_max": int(info.iters.max()),
           "converged": bool(info.converged.all()),
           "grad_finite": bool(torch.isfinite(dk).all())}
    if checks is not None:
        pick = sorted({0, 1, 2, int(info.iters.argmax())})

        def check():
            # the gradient again (untimed), with the oracle's FP64 targets, against the
            # oracle's reverse recursion at its own FP64 rollout
            from oracle import cma
            off = cma.uniform_offsets(B, T)
            yref = cma.Batch(p["topology"], kp_np, p["dt"], "rk4", d=d).rollout(p["s0"], off)
            yt = torch.tensor(yref, dtype=torch.float32, device=dev)
            dk2, _ = deer.deer_grad(dyn, s0, T, s, (2.0 * (s - yt)).contiguous(), prec="fp32",
                                    workspace=gws, stream=stream)
            dk2 = dk2.double().cpu().numpy()
            sub = cma.Batch(p["topology"][pick], p["params"][pick], p["dt"], "rk4", d=d)
            soff = cma.uniform_offsets(len(pick), T)
            sref = sub.rollout(p["s0"][pick], soff)
            yp = yref.reshape(B, T, d)[pick].reshape(-1, d)
            dk_ref, _ = sub.adjoint(p["s0"][pick], sref, 2.0 * (sref - yp), soff)
            sv = s.view(B, T, d)[torch.as_tensor(pick, device=dev)].reshape(-1, d).cpu().numpy()
            ferr = _rel_err_per_seq(sv, sref, soff)
            gerr = [float(np.max(np.abs(dk2[b] - dk_ref[i])) / np.max(np.abs(dk_ref[i])))
                    for i, b in enumerate(pick)]
            return {"max_rel_err_vs_oracle": float(ferr.max()),
                    "grad_max_rel_err_vs_oracle": max(gerr),
                    "oracle_sample": f"{len(pick)} of {B} trajectories (incl. the most Newton "
                                     "iterations): FP64 rollout and reverse adjoint in C"}
        checks.add(out, check)
    return out

def threshold_measurement(deer, N, lib, dev, stream, T=100000, d=32, gains=(0.5, 1.0, 2.0),
                          cap=300, checks=None):
    """The wall-clock side of the predictability threshold (Sec. ssc:exp_thresh): one
    mean-field RNN trajectory (B = 1, d = 32, W_ij ~ N(0, g^2/d), W_ii = 0, sinusoidal
    inputs) of length T, full-Jacobian DEER in FP32 (scaled residual 1e-5, sliding window,
    at most ``cap`` iterations) against the sequential GPU rollout (a warp walking the
    trajectory). Parallelising over time pays below the threshold (negative LLE, a few
    Newton iterations) and loses above it (positive LLE, iterations grow toward T)."""
    import numpy as np
    import torch
    import synth
    rows = []
    tuned = None
    for g in gains:
        p = synth.mean_field_rnn(1, T, d, g, seed=0)
        W = torch.tensor(p["W"], dtype=torch.float32, device=dev)
        dyn = deer.Dynamics.rnn_tanh(W)
        x = torch.tensor(p["x"].reshape(-1, d), dtype=torch.float32, device=dev)
        s0 = torch.tensor(p["s0"], dtype=torch.float32, device=dev)
        opts = dict(jac="full", tol=1e-5, prec="fp32", init="zeros", reset=True, window=True,
                    max_iters=cap)
        if tuned is None:
            # chunk length for a single long sequence, tuned once on the predictable case
            # (untimed): the per-sequence carry walks T / L chunk aggregates in order
            from paper_2603_16850_gb300 import autotune
            tuned = autotune.pick_best(
                (32, 64, 128, 256, 512),
                lambda L: _time_solve1(deer, dyn, s0, T, x, dict(opts, chunk=L), stream))
        opts["chunk"] = tuned["chunk"]
        ws_ = torch.empty(deer.deer_workspace_bytes(dyn, 1, T, **opts), dtype=torch.uint8,
                          device=dev)
        deer.deer_solve(dyn, s0, T, x, workspace=ws_, stream=stream, **opts)  # warm
        deer.deer_rollout(dyn, s0, T, x, prec="fp32", stream=stream)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        s, info = deer.deer_solve(dyn, s0, T, x, workspace=ws_, stream=stream, **opts)
        e[1].record(stream)
        e[2].record(stream)
        ref = deer.deer_rollout(dyn, s0, T, x, prec="fp32", stream=stream)
        e[3].record(stream)
        torch.cuda.synchronize()
        deer_ms, seq_ms = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
        # one more solve with the library's per-phase events (not the timed one)
        lib.deer_profile_reset()
        lib.deer_profile_enable(1)
        deer.deer_solve(dyn, s0, T, x, workspace=ws_, stream=stream, **opts)
        torch.cuda.synchronize()
        lib.deer_profile_enable(0)
        prof = N.deer_profile()
        lib.deer_profile_read(prof)
        lle = float(deer.deer_lle(dyn, s0, T, ref, x=x, prec="fp32", stream=stream)[0])
        err = float((s - ref).abs().max() / ref.abs().max())
        row = {"g": g, "lle": lle, "newton_iters": int(info.iters[0]),
               "converged": bool(info.converged[0]), "deer_ms": deer_ms,
               "sequential_ms": seq_ms, "speedup": seq_ms / deer_ms,
               "max_rel_diff_vs_gpu_rollout": err,
               "phase_ms": {n: prof.ms[i] for i, n in enumerate(N.PHASES)}}
        rows.append(row)
        if checks is not None:
            s_host = s.cpu().numpy()

            def check(p=p, s_host=s_host):
                from oracle import dynamics as odyn
                from oracle import newton as onewton
                r = onewton.rollout(odyn.MeanFieldRNN(p["W"], p["x"]), p["s0"], T)[0]
                e = _rel_err_per_seq(s_host, r, [0, T])
                return {"max_rel_err_vs_oracle": float(e.max())}
            checks.add(row, check)
    return {"workload": f"mean-field RNN d={d}, B=1, T={T}, FP32 DEER (cap {cap} "
                        "iterations) vs sequential GPU rollout",
            "chunk": {"chosen": tuned["chunk"], "tuning_ms": tuned["timings"],
                      "how": "autotune.pick_best on the g=%.1f problem" % gains[0]},
            "rows": rows}


def _time_solve1(deer, dyn, s0, T, x, opts, stream):
    """Milliseconds of one solve of B sequences of length T (after one warm-up)."""
    import torch
    deer.deer_solve(dyn, s0, T, x, stream=stream, **opts)
    torch.cuda.synchronize()
    e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    e0.record(stream)
    deer.deer_solve(dyn, s0, T, x, stream=stream, **opts)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def dyn_sub(deer, p, d, dev, n=32):
    """Kinetics of the first n systems of a problem (autotuning subset)."""
    import torch
    return deer.Dynamics.massaction(
        torch.tensor(p["topology"][:n], dtype=torch.int32, device=dev),
        torch.tensor(p["params"][:n], dtype=torch.float64, device=dev), d, p["dt"])


def _time_solve(deer, dyn, s0, offsets, opts, stream):
    """Milliseconds of one batched solve (after one warm-up), CUDA events."""
    import torch
    deer.deer_solve_batched(dyn, s0, offsets, stream=stream, **opts)
    torch.cuda.synchronize()
    e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    e0.record(stream)
    deer.deer_solve_batched(dyn, s0, offsets, stream=stream, **opts)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def ragged_mixed_measurement(deer, N, lib, dev, stream, B=10000, group=1000, checks=None,
                             jac_bytes_max=8 << 30):
    """Ragged mixed-precision workload: B = 10000 d=16 kinetic networks (24 reactions),
    lengths uniform on [1000, 100000] (sum T ~ 5e8), RK4 dt=1e-3, bf16 Jacobians with
    float32 scan accumulation, float64 state and residual, in ONE deer_solve_batched call:
    the bf16 Jacobians of all rows (256 GB) exceed the bound, so none is stored (each chunk's
    aggregate is formed while it is linearised; the scan's final pass linearises again).
    The first `group` sequences are also solved on their own with the stored-Jacobian mixed
    path and by plain FP32 parallel Newton, and the whole batch by the sequential GPU
    rollout, for comparison."""
    import numpy as np
    import torch
    import synth
    d, R = 16, 24
    lengths = synth.ragged_lengths(B, 1000, 100000, seed=5)
    off = synth.offsets_from_lengths(lengths)
    p = synth.massaction(B, d, R, 1, seed=6)
    topo = torch.tensor(p["topology"], dtype=torch.int32, device=dev)
    k = torch.tensor(p["params"], dtype=torch.float64, device=dev)
    s0 = torch.tensor(p["s0"], dtype=torch.float64, device=dev)
    dyn = deer.Dynamics.massaction(topo, k, d, p["dt"])
    # scaled residual 1e-12: the residual left at convergence adds up along the conserved
    # directions over up to 1e5 steps (1e-10 leaves errors of 1e-7 against the rollout)
    opts = dict(jac="full", tol=1e-12, prec="mixed_bf16", init="zeros", reset=True,
                window=True)
    # chunk length chosen by the autotuner on a 32-trajectory subset of the same
    # distribution (not timed), then used for the whole batch
    from paper_2603_16850_gb300 import autotune
    sub_off = off[:33] - off[0]
    t0 = time.perf_counter()
    timings = autotune.pick_best(
        (32, 64, 128, 256),
        lambda L: _time_solve(deer, dyn_sub(deer, p, d, dev), s0[:32].contiguous(), sub_off,
                              dict(opts, chunk=L), stream))
    tune_s = time.perf_counter() - t0
    opts["chunk"] = timings["chunk"]
    ntot = int(off[-1])
    big = dict(opts, jac_bytes_max=jac_bytes_max)
    nbytes = deer.deer_workspace_bytes(dyn, B, ntot, **big)
    ws_ = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    lib.deer_profile_reset()
    lib.deer_profile_enable(1)
    e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    e0.record(stream)
    s, info = deer.deer_solve_batched(dyn, s0, off, workspace=ws_, stream=stream, **big)
    e1.record(stream)
    torch.cuda.synchronize()
    lib.deer_profile_enable(0)
    prof = N.deer_profile()
    lib.deer_profile_read(prof)
    ms = e0.elapsed_time(e1)
    del ws_
    # comparisons on the first `group` sequences: the stored-Jacobian mixed path, plain
    # FP32 parallel Newton (float32 Jacobians, scan, residual and state, no compensation;
    # tol 5e-7 twice); and the sequential GPU rollout of the whole batch in float64 and
    # float32
    goff = off[:group + 1]
    gtot = int(goff[-1])
    gdyn = dyn_sub(deer, p, d, dev, n=group)
    gs0 = s0[:group].contiguous()
    wsg = torch.empty(deer.deer_workspace_bytes(gdyn, group, gtot, **opts), dtype=torch.uint8,
                      device=dev)
    deer.deer_solve_batched(gdyn, gs0, goff, workspace=wsg, stream=stream, **opts)  # warm
    torch.cuda.synchronize()
    e0.record(stream)
    _, ginfo = deer.deer_solve_batched(gdyn, gs0, goff, workspace=wsg, stream=stream, **opts)
    e1.record(stream)
    torch.cuda.synchronize()
    gms = e0.elapsed_time(e1)
    del wsg
    gdyn32 = deer.Dynamics.massaction(gdyn.topology, gdyn.params.float(), d, p["dt"])
    gs032 = gs0.float()
    o32 = dict(jac="full", tol=5e-7, confirm=2, prec="fp32", init="zeros", reset=True,
               compensate=False, window=True, chunk=opts["chunk"])
    ws32 = torch.empty(deer.deer_workspace_bytes(gdyn32, group, gtot, **o32), dtype=torch.uint8,
                       device=dev)
    deer.deer_solve_batched(gdyn32, gs032, goff, workspace=ws32, stream=stream, **o32)  # warm
    torch.cuda.synchronize()
    e0.record(stream)
    s32, info32 = deer.deer_solve_batched(gdyn32, gs032, goff, workspace=ws32, stream=stream,
                                          **o32)
    e1.record(stream)
    torch.cuda.synchronize()
    ms32 = e0.elapsed_time(e1)
    del ws32
    off_d = torch.tensor(off, dtype=torch.int64, device=dev)
    dyn32 = deer.Dynamics.massaction(topo, k.float(), d, p["dt"])
    roll = {}
    for name, dd, ss in (("fp64", dyn, s0), ("fp32", dyn32, s0.float())):
        deer.deer_rollout(dd, ss, 0, offsets=off_d, prec=name, stream=stream)
        torch.cuda.synchronize()
        e0.record(stream)
        deer.deer_rollout(dd, ss, 0, offsets=off_d, prec=name, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        roll[name] = e0.elapsed_time(e1)
    lin_rows = prof.rows[1]
    lin_s = prof.ms[1] / 1000.0
    out = {"workload": f"ragged mass action d=16 R=24, T ~ U[1000,100000], B={B} in one call "
                       "(sum T = %d), bf16 Jacobians recomputed (not stored) / fp32 scan / "
                       "fp64 residual, tol 1e-12" % ntot,
           "chunk": {"chosen": timings["chunk"], "tuning_s": tune_s,
                     "how": "autotune.pick_best on 32 trajectories"},
           "jac_bytes_max": jac_bytes_max, "workspace_bytes": int(nbytes),
           "rows_linearized_pass1": int(lin_rows), "rows_scanned": int(prof.rows[3]),
           "linearize_rows_per_s": lin_rows / max(lin_s, 1e-12),
           "total_steps": ntot, "ms": ms, "value": ntot / (ms / 1000.0), "unit": UNIT,
           "newton_iters_max": int(info.iters.max()),
           "newton_iters_p50": float(np.percentile(info.iters.numpy(), 50)),
           "converged": bool(info.converged.all()),
           "phase_ms": {n: prof.ms[i] for i, n in enumerate(N.PHASES)},
           "group_stored_jacobians": {"B": group, "total_steps": gtot, "ms": gms,
                                      "value": gtot / (gms / 1000.0), "unit": UNIT,
                                      "newton_iters_max": int(ginfo.iters.max())},
           "fp32_newton": {"B": group, "ms": ms32, "value": gtot / (ms32 / 1000.0),
                           "unit": UNIT, "newton_iters_max": int(info32.iters.max()),
                           "converged": bool(info32.converged.all()),
                           "note": "float32 everything on the first group: its fixed point "
                                   "is the float32 rollout, not the float64 one"},
           "sequential_gpu_rollout": {name: {"ms": v, "value": ntot / (v / 1000.0),
                                             "unit": UNIT} for name, v in roll.items()}}
    if checks is not None:
        lengths_a = np.diff(off)
        pick = sorted(set(np.argsort(-lengths_a)[:4].tolist()) |
                      set(np.argsort(-info.iters.numpy())[:4].tolist()) | set(range(24)))
        rows_of = [np.arange(off[b], off[b + 1]) for b in pick]
        idx = torch.as_tensor(np.concatenate(rows_of), device=dev)
        s_host = s[idx].cpu().numpy()
        gpick = [b for b in pick if b < group]
        grows = [np.arange(off[b], off[b + 1]) for b in gpick]
        s32_host = s32[torch.as_tensor(np.concatenate(grows), device=dev)].double().cpu().numpy()
        sub_off2 = np.concatenate([[0], np.cumsum([len(r) for r in rows_of])])
        g_off2 = np.concatenate([[0], np.cumsum([len(r) for r in grows])])

        def check():
            from oracle import cma
            sub = cma.Batch(p["topology"][pick], p["params"][pick], p["dt"], "rk4", d=d)
            ref = sub.rollout(p["s0"][pick], sub_off2)
            err = _rel_err_per_seq(s_host, ref, sub_off2)
            gsel = [pick.index(b) for b in gpick]
            gref = np.concatenate([ref[sub_off2[i]:sub_off2[i + 1]] for i in gsel])
            err32 = _rel_err_per_seq(s32_host, gref, g_off2)
            out["fp32_newton"]["max_rel_err_vs_oracle"] = float(err32.max())
            return {"max_rel_err_vs_oracle": float(err.max()),
                    "oracle_sample": f"{len(pick)} of {B} trajectories (the 4 longest, the 4 "
                                     "with the most iterations, the first 24), FP64 rollout "
                                     "in C"}
        checks.add(out, check)
    return out
def compose_measurement(deer, N, lib, dev, stream, B=1000):
    """The chunk products of the dense scan on the tensor cores, in both forms: the d = 16
    mixed-precision chunk pass as warp-level bf16 MMAs (one chunk per warp, every
    multiply-add useful) and as tcgen05 MMAs (8 chunks per CTA stacked block-diagonally,
    accumulator in tensor memory, 1/8 useful), timed on the ragged d = 16 group with stored
    Jacobians; and the d = 32 float32 chunk pass as warp-level tf32 MMAs (three-term split)
    against the SIMT pass, on the single-trajectory RNN (T = 1e5). Scan-phase device time
    from the library's CUDA events; the chunk passes' share and their tensor-pipe busy
    fractions come from the ncu captures under profiles/."""
    import numpy as np
    import torch
    import synth
    d, R = 16, 24
    lengths = synth.ragged_lengths(B, 1000, 100000, seed=5)
    off = synth.offsets_from_lengths(lengths)
    p = synth.massaction(B, d, R, 1, seed=6)
    dyn = dyn_sub(deer, p, d, dev, n=B)
    s0 = torch.tensor(p["s0"], dtype=torch.float64, device=dev)
    opts = dict(jac="full", tol=1e-12, prec="mixed_bf16", init="zeros", reset=True,
                window=True, chunk=128)
    ws_ = torch.empty(deer.deer_workspace_bytes(dyn, B, int(off[-1]), **opts),
                      dtype=torch.uint8, device=dev)
    out = {"mixed_d16": {"workload": f"ragged mass action d=16, B={B}, stored bf16 Jacobians"}}
    try:
        for mode, name in ((1, "warp_mma_bf16"), (2, "tcgen05_block_diagonal")):
            deer.set_tensor_cores(mode)
            deer.deer_solve_batched(dyn, s0, off, workspace=ws_, stream=stream, **opts)
            torch.cuda.synchronize()
            lib.deer_profile_reset()
            lib.deer_profile_enable(1)
            e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
            e0.record(stream)
            _, info = deer.deer_solve_batched(dyn, s0, off, workspace=ws_, stream=stream, **opts)
            e1.record(stream)
            torch.cuda.synchronize()
            lib.deer_profile_enable(0)
            prof = N.deer_profile()
            lib.deer_profile_read(prof)
            out["mixed_d16"][name] = {"ms": e0.elapsed_time(e1), "scan_ms": prof.ms[3],
                                      "rows_scanned": int(prof.rows[3]),
                                      "newton_iters_max": int(info.iters.max())}
        del ws_
        T, dr = 100000, 32
        pr = synth.mean_field_rnn(1, T, dr, 0.5, seed=0)
        rd = deer.Dynamics.rnn_tanh(torch.tensor(pr["W"], dtype=torch.float32, device=dev))
        x = torch.tensor(pr["x"].reshape(-1, dr), dtype=torch.float32, device=dev)
        s0r = torch.tensor(pr["s0"], dtype=torch.float32, device=dev)
        ro = dict(jac="full", tol=1e-5, prec="fp32", init="zeros", reset=True, window=True,
                  chunk=256)
        out["dense_d32"] = {"workload": "mean-field RNN d=32, B=1, T=1e5, FP32"}
        for mode, name in ((1, "warp_mma_tf32x3"), (0, "simt_ring4")):
            deer.set_tensor_cores(mode)
            deer.deer_solve(rd, s0r, T, x, stream=stream, **ro)
            torch.cuda.synchronize()
            lib.deer_profile_reset()
            lib.deer_profile_enable(1)
            e0.record(stream)
            _, info = deer.deer_solve(rd, s0r, T, x, stream=stream, **ro)
            e1.record(stream)
            torch.cuda.synchronize()
            lib.deer_profile_enable(0)
            prof = N.deer_profile()
            lib.deer_profile_read(prof)
            out["dense_d32"][name] = {"ms": e0.elapsed_time(e1), "scan_ms": prof.ms[3],
                                      "newton_iters": int(info.iters.max())}
    finally:
        deer.set_tensor_cores(1)
    return out


def dense_elk_measurement(deer, dev, stream, B=4, d=8, lam=1.0, iters=10):
    """Cost of one dense-ELK iteration (full-Jacobian Kalman-filter step, Sec. 4.2-4.3)
    against one undamped DEER iteration on the same few long sequences (mass action d=8,
    RK4, FP64, reset heuristic on: undamped DEER overflows on these horizons; fixed
    iteration count, tol 0). With chunks of 128 rows the covariance
    recursion runs in parallel over time (chunk elements, carry, per-chunk restart); with
    chunks of T/4 rows (T = 4096, chunk 1024) the library keeps one covariance chain per
    sequence, which shows what the parallel form saves. The paper's own figures for the
    ratio: 3.6 ms per ELK step against 0.282 ms per DEER step."""
    import torch
    import synth
    R = {8: 12, 16: 24}[d]
    out = {}
    for T, chunks in ((65536, (128,)), (4096, (128, 1024))):
        p = synth.massaction(B, d, R, T, seed=80, dt=0.01)
        dyn = deer.Dynamics.massaction(
            torch.tensor(p["topology"], dtype=torch.int32, device=dev),
            torch.tensor(p["params"], dtype=torch.float64, device=dev), d, p["dt"])
        s0 = torch.tensor(p["s0"], dtype=torch.float64, device=dev)
        for chunk in chunks:
            row = {}
            for name, extra in (("deer", {}), ("elk", dict(damp="elk", damp_param=lam))):
                opts = dict(jac="full", tol=0.0, max_iters=iters, init="s0", prec="fp64",
                            chunk=chunk, reset=True, **extra)
                ms = _time_solve1(deer, dyn, s0, T, None, opts, stream)
                row[name + "_ms_per_iter"] = ms / iters
            row["elk_over_deer"] = row["elk_ms_per_iter"] / row["deer_ms_per_iter"]
            row["covariance"] = ("parallel over time" if T // chunk >= 8
                                 else "one chain per sequence")
            out["T%d_chunk%d" % (T, chunk)] = row
    out["paper_elk_over_deer"] = 3.6 / 0.282
    return {"workload": f"mass action d={d} RK4 FP64, B={B}, lambda={lam}, "
                        f"{iters} iterations (tol 0)", **out}


def run_only(args):
    """One secondary workload alone, for profiler captures of its kernels."""
    import torch

    import paper_2603_16850_gb300 as deer
    from paper_2603_16850_gb300 import _native as N
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    lib = N.load()
    if args.only == "gru":
        out = gru_diag_measurement(deer, N, lib, dev, stream, steps=max(args.steps, 1),
                                   B=args.batch or 64)
    elif args.only == "ragged_mixed":
        out = ragged_mixed_measurement(deer, N, lib, dev, stream, B=args.batch or 10000,
                                       group=min(1000, args.batch or 1000))
    elif args.only == "brusselator":
        out = brusselator_measurement(deer, dev, stream, N=N, lib=lib)
    elif args.only == "gru_window":
        out = gru_diag_measurement(deer, N, lib, dev, stream, steps=max(args.steps, 1),
                                   B=args.batch or 64, window=True)
    elif args.only == "gru_elk":
        out = gru_elk_measurement(deer, dev, stream, B=args.batch or 64)
    elif args.only == "dense_elk":
        out = dense_elk_measurement(deer, dev, stream, B=args.batch or 4)
    elif args.only == "compose":
        out = compose_measurement(deer, N, lib, dev, stream, B=args.batch or 1000)
    elif args.only == "threshold":
        gains = tuple(float(v) for v in args.gains.split(",")) if args.gains else (0.5, 1.0, 2.0)
        out = threshold_measurement(deer, N, lib, dev, stream, gains=gains)
    else:
        out = adjoint_measurement(deer, N, lib, dev, stream, B=args.batch or 256)
    print(json.dumps({"only": args.only, **out}), flush=True)
    return 0


_ALU_PEAKS = {}


def _alu_peaks(lib, dev):
    """Peak rates of this GPU measured by the library's own microbenchmarks
    (deer_measure_peak: FP32 and FP64 FMA on every SM, dense tcgen05 MMAs of kind::tf32 and
    kind::f16 with bf16 operands), in TFLOP/s, timed with CUDA events; the SM count comes
    from the device. Falls back to SM count x 128 FP32 lanes x 2 x the maximum SM clock
    where the library has no microbenchmark."""
    if _ALU_PEAKS:
        return _ALU_PEAKS
    import torch
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks, _ = _peaks()
    if hasattr(lib, "deer_measure_peak"):
        out = C.c_double(0.0)
        for name, what in (("fp32", 0), ("fp64", 1), ("tf32_tc", 2), ("bf16_tc", 3)):
            st = lib.deer_measure_peak(what, torch.cuda.current_stream().cuda_stream,
                                       C.byref(out))
            if st == 0 and out.value > 0:
                _ALU_PEAKS[name] = out.value / 1e12
                _ALU_PEAKS[name + "_source"] = "measured (deer_measure_peak)"
    if "fp32" not in _ALU_PEAKS:
        mhz = peaks.get("sm_max_mhz", 2070.0)
        _ALU_PEAKS["fp32"] = sms * 128 * 2 * mhz * 1e6 / 1e12
        _ALU_PEAKS["fp32_source"] = f"derived: {sms} SMs x 128 lanes x 2 flop x {mhz:.0f} MHz"
    _ALU_PEAKS["sms"] = sms
    return _ALU_PEAKS


def _tf32_peak(lib, peaks):
    """tf32 tensor-pipe peak: measured when the library's microbenchmark ran, else the
    measured bf16 peak x the nominal tf32 / bf16 ratio (1.1 / 2.25 PFLOP/s dense)."""
    if "tf32_tc" in _ALU_PEAKS:
        return _ALU_PEAKS["tf32_tc"], _ALU_PEAKS["tf32_tc_source"]
    _, kind = _peaks()
    return peaks["bf16_tflops"] * 1.1 / 2.25, f"bf16 {kind} x 1.1/2.25 nominal"


def run(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2603_16850_gb300 as deer
    from paper_2603_16850_gb300 import _native as N

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    w = dict(WORKLOAD)
    if args.batch:
        w["B"] = args.batch
    B, d, T = w["B"], w["d"], w["T"]
    p = _problem(rank, w["B"])
    k = torch.tensor(p["params"], dtype=torch.float32, device=dev)
    topo = torch.tensor(p["topology"], dtype=torch.int32, device=dev)
    s0 = torch.tensor(p["s0"], dtype=torch.float32, device=dev)
    dyn = deer.Dynamics.massaction(topo, k, d, w["dt"], w["integrator"])
    opts = dict(jac="full", tol=w["tol"], confirm=w["confirm"], prec="fp32", init=w["init"],
                reset=True, window=w["window"])
    nbytes = deer.deer_workspace_bytes(dyn, B, B * T, **opts)
    workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    lib = N.load()

    def step():
        return deer.deer_solve(dyn, s0, T, stream=stream, workspace=workspace, **opts)

    for _ in range(args.warmup):
        s, info = step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # raw nvidia-smi samples go to DEER_CLOCKS_DIR (default: the system temporary
    # directory); the JSON line carries their summary
    clocks_dir = os.environ.get("DEER_CLOCKS_DIR", tempfile.gettempdir())
    clocks = Clocks(local, os.path.join(clocks_dir, f"deer_clocks_rank{rank}.csv"))
    lib.deer_profile_reset()
    lib.deer_profile_enable(1)
    launches0 = lib.deer_kernel_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    iters = []
    for _ in range(args.steps):
        s, info = step()
        iters.append(int(info.iters.max()))
        if not bool(info.converged.all()):
            raise RuntimeError("solve did not converge")
    ev1.record(stream)
    torch.cuda.synchronize()
    lib.deer_profile_enable(0)
    launches = lib.deer_kernel_launch_count() - launches0
    prof = N.deer_profile()
    lib.deer_profile_read(prof)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = _max_over_ranks(ms, dev)
    value = _whole_job_rate(B * T, ws, ms)

    # roofline of the dominant kernel, the fused iteration kernel (apply the pending scan
    # step, linearise, form the chunk aggregates; launches and times from the library's
    # per-phase CUDA events on the solver's stream): the algorithmic work the measurement
    # plan fixes per row (4524 flop, 96 B with A kept on chip) against the measured peaks.
    peaks, peak_kind = _peaks()
    alu = _alu_peaks(lib, dev)
    n_lin = max(prof.launches[1], 1)
    lin_ms = prof.ms[1] / n_lin
    lin_rows = prof.rows[1] / n_lin
    alu_ach = lin_rows * ALGO_FLOP_PER_ROW / (lin_ms / 1000.0) / 1e12
    hbm_ach = lin_rows * ALGO_BYTES_PER_ROW / (lin_ms / 1000.0) / 1e9
    impl_gbs = lin_rows * IMPL_BYTES_PER_ROW / (lin_ms / 1000.0) / 1e9
    alu_frac, hbm_frac = alu_ach / alu["fp32"], hbm_ach / peaks["hbm_gbs"]
    traffic = FUSED_TRAFFIC_PER_ROW * lin_rows if FUSED_TRAFFIC_PER_ROW else None
    roof = {"kernel": "k_fused_ma_lps<float,8,RK4>", "bound": "alu", "achieved": alu_ach,
            "peak": alu["fp32"], "unit": "TFLOP/s", "frac": alu_frac, "traffic": traffic,
            "peak_source": "FP32 FMA, " + alu["fp32_source"],
            "flop_per_row": ALGO_FLOP_PER_ROW, "algorithmic_bytes_per_row": ALGO_BYTES_PER_ROW,
            "hbm_frac_algorithmic": hbm_frac, "hbm_peak_gbs": peaks["hbm_gbs"],
            "hbm_peak_source": peak_kind,
            "impl_bytes_per_row": IMPL_BYTES_PER_ROW, "impl_gbs": impl_gbs,
            "traffic_per_row": FUSED_TRAFFIC_PER_ROW,
            "traffic_ratio": (FUSED_TRAFFIC_PER_ROW / ALGO_BYTES_PER_ROW
                              if FUSED_TRAFFIC_PER_ROW else None),
            "traffic_source": "ncu dram bytes per row (profiles/, B=512) x rows per launch",
            "launches": int(prof.launches[1]), "avg_launch_ms": lin_ms,
            "avg_rows_per_launch": lin_rows,
            "share_of_step": prof.ms[1] / max(sum(prof.ms), 1e-9)}
    for key in ("fp64", "tf32_tc", "bf16_tc"):
        if key in alu:
            roof["measured_peak_" + key + "_tflops"] = alu[key]

    # sequential GPU rollout (comparison baseline), same precision
    for _ in range(2):
        deer.deer_rollout(dyn, s0, T, prec="fp32")
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nroll = 3
    for _ in range(nroll):
        deer.deer_rollout(dyn, s0, T, prec="fp32", stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    roll_ms = e0.elapsed_time(e1) / nroll

    # end to end through the public API with pinned host buffers
    k_h = k.cpu().pin_memory()
    topo_h = topo.cpu().pin_memory()
    s0_h = s0.cpu().pin_memory()
    dyn_h = deer.Dynamics.massaction(topo_h, k_h, d, w["dt"], w["integrator"])
    # the trajectory comes back into one pinned host buffer allocated up front (pinning
    # 2.1 GB costs more than copying it)
    out_h = torch.empty((B * T, d), dtype=torch.float32, pin_memory=True)
    deer.deer_solve(dyn_h, s0_h, T, workspace=workspace, out=out_h, **opts)
    torch.cuda.synchronize()
    n_e2e = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        s_h, _ = deer.deer_solve(dyn_h, s0_h, T, workspace=workspace, out=out_h, **opts)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / n_e2e
    h2d = k_h.numel() * 4 + topo_h.numel() * 4 + s0_h.numel() * 4
    d2h = s_h.numel() * 4
    s_head = s.cpu().numpy()
    del workspace

    extra = {}
    checks = OracleChecks() if not args.no_cpu_baseline else None
    if rank == 0 and ws == 1 and not args.no_extra:
        gru_cache = {}
        extra["lle"] = lle_measurement(deer, dyn, s0, s, T, d, stream)
        extra["brusselator"] = brusselator_measurement(deer, dev, stream, checks=checks, N=N,
                                                       lib=lib)
        extra["gru_quasi_deer"] = gru_diag_measurement(deer, N, lib, dev, stream, checks=checks,
                                                       gru_cache=gru_cache)
        extra["gru_quasi_elk"] = gru_elk_measurement(deer, dev, stream, checks=checks,
                                                     gru_cache=gru_cache)
        extra["adjoint"] = adjoint_measurement(deer, N, lib, dev, stream, checks=checks)
        extra["ragged_mixed"] = ragged_mixed_measurement(deer, N, lib, dev, stream,
                                                         checks=checks)
        extra["threshold"] = threshold_measurement(deer, N, lib, dev, stream, checks=checks)
        q = extra["gru_quasi_deer"]
        roof["diag_scan_kernel"] = q["diag_scan"]["kernel"]
        roof["diag_scan_gbs"] = q["diag_scan"]["achieved"]
        roof["diag_scan_frac"] = q["diag_scan"]["frac"]
        roof["diag_scan_peak_source"] = q["diag_scan"]["peak_source"]
        if "tensor_frac" in q["linearize"]:
            roof["gru_lin_tc_tensor_frac"] = q["linearize"]["tensor_frac"]

    # CPU-baseline leg: the FP64 oracle timed on the host cores (the whole workload's
    # sequential rollout, in plain C, split over every core), then every GPU result of this
    # run compared with the oracle
    cpu = None
    head_err = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ref, cpu_s, threads = cpu_oracle_rollout(p)
        cpu = {"value": B * T / cpu_s, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"the whole workload ({B} trajectories x {T} steps): FP64 sequential "
                         f"rollout in plain C on {threads} host threads, {cpu_s:.2f} s"}
        head_err = float(_rel_err_per_seq(s_head, ref, np.arange(B + 1) * T).max())
        del ref
        checks.run()

    if rank == 0:
        summary = {"max_rel_err_vs_oracle": head_err}
        for name, e in extra.items():
            if "value" in e:
                summary[name + "_value"] = e["value"]
            if "max_rel_err_vs_oracle" in e:
                summary[name + "_max_rel_err_vs_oracle"] = e["max_rel_err_vs_oracle"]
        if "adjoint" in extra:
            a = extra["adjoint"]
            summary["adjoint_forward_ms"] = a["forward_ms"]
            summary["adjoint_grad_ms"] = a["grad_ms"]
            if "grad_max_rel_err_vs_oracle" in a:
                summary["adjoint_grad_max_rel_err_vs_oracle"] = a["grad_max_rel_err_vs_oracle"]
        if "gru_quasi_deer" in extra:
            summary["diag_scan_frac_of_hbm"] = extra["gru_quasi_deer"]["diag_scan"]["frac"]
        if "ragged_mixed" in extra:
            summary["ragged_mixed_fp32_newton_max_rel_err_vs_oracle"] = \
                extra["ragged_mixed"]["fp32_newton"].get("max_rel_err_vs_oracle")
        if "gru_quasi_elk" in extra:
            summary["gru_quasi_elk_max_rel_err_vs_oracle"] = max(
                (r.get("max_rel_err_vs_oracle", 0.0) for r in extra["gru_quasi_elk"]["sweep"]),
                default=None)
        if "threshold" in extra:
            for r in extra["threshold"]["rows"]:
                summary[f"threshold_g{r['g']}_speedup_vs_sequential"] = r["speedup"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": CONFIG_NAME, "B_per_gpu": B, "T": T, "d": d, "reactions": 12,
                       "tol": w["tol"], "confirm": w["confirm"], "init": w["init"],
                       "reset": True, "sliding_window": w["window"],
                       "compensated_state": True,
                       "newton_iters_max": iters[-1],
                       "newton_iters_p50": float(np.percentile(info.iters.numpy(), 50)),
                       "newton_iters_p99": float(np.percentile(info.iters.numpy(), 99)),
                       "l2": "working set (Jacobians 17 GB) far larger than L2; no flush needed",
                       "parallelism": f"replicas x{ws}"},
            "gpu_launches": int(launches),
            "max_rel_err_vs_oracle": head_err,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": ws * B * T / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "sequential_gpu_rollout": {"value": ws * B * T / (roll_ms / 1000.0), "unit": UNIT,
                                       "ms": roll_ms},
            "phase_ms_per_step": {n: prof.ms[i] / args.steps for i, n in enumerate(N.PHASES)},
            "clocks": clk,
            **extra,
            # last, so that the end of the line (what a truncated log keeps) holds the
            # secondary results and their errors against the oracle
            "summary": summary,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the secondary GRU quasi-DEER measurement")
    ap.add_argument("--only", default="", choices=["", "brusselator", "gru", "gru_window",
                                                   "gru_elk", "adjoint", "ragged_mixed",
                                                   "threshold", "compose", "dense_elk"],
                    help="run one secondary workload alone (with --batch) and print it")
    ap.add_argument("--gains", default="",
                    help="--only threshold: comma-separated RNN gains g (default 0.5,1.0,2.0)")
    ap.add_argument("--batch", type=int, default=0,
                    help="trajectories per GPU (default 4096; smaller for profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
