#!/usr/bin/env python3
"""Benchmark of the split time step (transport + RK2[C + precession] + transport).

Default workload (plain FP64 at scale): N = 64 velocity points per dimension,
Nx = 128 cells, Dirichlet walls (Fermi-Dirac beta = 1, mu = 0, U = 1),
B = (0, 0, 0.5), dt = 0.005, J = M = 32, L = 12, R = 7.5, seeded synthetic
Fermi-Dirac-perturbed state (5 % Hermitian perturbation).  One step = one
split time step of all 128 cells = 2 collision-operator evaluations.

Prints one JSON line (rank 0).  Metric: C[W] cell*k-pts/s
(= 2 * Nx * N^2 collision evaluations per step / time).  At N = 1 the line's
"forms" object carries the rest of the metric on the same 64 x 64, Nx = 128
grid: the FP32-split form of the workload (steps/s, C[W] cell*k-pts/s, its
error against the FP64 GPU form and the stored oracle cells, stated
tolerances) and the adjoint/forward time ratio of the differentiation
configuration over a short horizon (--forms-horizon, default 2 split steps),
with the forward keeping every intermediate state (full tape) and, beside it,
with a checkpoint every step recomputed by the reverse sweep.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --mode collide [--cells C]   # time C[W] alone on the first C cells
  python bench.py --mode vjp [--cells C]       # time the collision VJP alone
  python bench.py --mode peaks                 # measured FP64 / FP32 arithmetic issue rates

--mode collide (not the benchmark line; used for profiling) times only the
collision operator, one evaluation of the first C cells per step.

--impl reference times the FP64 CPU oracle (the baseline: no other
implementation of this method exists) on the host cores, one cell's C[W] per
step, on the same workload.  Under torchrun with N > 1, "ours" runs independent
replicas (one full simulation per GPU, weak scaling); "reference" runs on rank 0
only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 152
FP64_FMA_PER_CLK_PER_SM = 2          # GB300: measured 2.00 DFMA lanes/clk/SM (bench.py --mode peaks)
FP32_FMA_PER_CLK_PER_SM = 128        # measured 122 FFMA lanes/clk/SM (the same run)
# DRAM bytes (read + write) per (cell, j, m) unit of the default I3 kernel from one ncu capture of a
# slice (8 cells at N = 64: k_i3_sf in FP64, k_i3_wl in FP32; 4 cells at N = 128: k_i3_cluster in its
# register-accumulating shape), scaled by units; absent for sizes with no capture of the current kernel.
I3_DRAM_BYTES_PER_UNIT = {(64, 0): 113.013e9 / 8192, (64, 1): 3.090e9 / 8192, (128, 1): 15.160e9 / 4096}
# The same for the default I3 transpose kernel (8 cells at N = 64: k_i3_vjp_wl, one cotangent).
I3_VJP_DRAM_BYTES_PER_UNIT = {(64, 1): 5.463e9 / 8192}


def workload(name="plain_fp64_n64", precision=None):
    from paper_1408_1782_gb300 import inputs
    wl = dict(inputs.WORKLOADS[name])
    wl["name"] = name
    if precision is not None:
        wl["precision"] = precision
    return wl


def i3_flops_per_unit(N):
    """Algorithmic FLOPs of one (cell, j, m) unit of the I3 (Hu-Ying) term, FFT convention:
    36 real 2-D transforms of P = (2N)^2 points at 2.5 P log2 P each (4 shifts, 16 forward,
    16 inverse) plus 67 P pointwise flops (16 products, 16 psi' scalings of complex spectra,
    16 multiply-adds, the shift phases)."""
    P = (2 * N) ** 2
    return 90.0 * P * math.log2(P) + 67.0 * P


# ---------------------------------------------------------------------------
# CPU side (the oracle): a bounded sample on the host cores
# ---------------------------------------------------------------------------

def oracle_sample(wl, ncores, repeats=1, warmup=0):
    """Time the oracle's C[W] for one cell of the workload (its 60 independent integral
    terms spread over `ncores` spawned processes).  Returns (seconds per sample, cores)."""
    import multiprocessing as mp

    import numpy as np

    from oracle import qbe_oracle as O
    from paper_1408_1782_gb300 import inputs

    p = O.Params(N=wl["N"], L=wl["L"], R=wl["R"], J=wl["J"], M=wl["M"])
    W = inputs.synthetic_w(wl["N"], wl["Nx"], L=wl["L"], seed=0, perturb=wl["perturb"])
    cell = np.ascontiguousarray(W[:1])
    ctx = mp.get_context("spawn")
    times = []
    with ctx.Pool(ncores) as pool:
        mapper = lambda f, it: pool.map(f, list(it), chunksize=1)
        small = O.Params(N=8, J=2, M=1)
        for _ in range(warmup):                           # untimed; numpy has nothing to warm up
            O.collision(inputs.synthetic_w(8, 1, seed=1), small, mapper=mapper)
        for _ in range(repeats):
            t = time.perf_counter()
            O.collision(cell, p, mapper=mapper)
            times.append(time.perf_counter() - t)
    return times, ncores


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = workload(args.workload, args.precision)
    ncores = min(16, host_cores())
    times, cores = oracle_sample(wl, ncores, repeats=args.steps, warmup=args.warmup)
    T = sum(times)
    npts = wl["N"] ** 2
    value = args.steps * npts / T
    sample = (f"per step: C[W] of 1 of the {wl['Nx']} cells (N={wl['N']}, J=M={wl['J']}), the oracle's "
              f"60 integral terms on {cores} spawned processes")
    line = {
        "impl": "reference", "metric": "C[W] cell·k-pts/s", "value": value, "unit": "cell·k-pts/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Fermi-Dirac-perturbed W)", "impl_note": "FP64 CPU oracle",
        "config": config_dict(wl, args.gpus),
        "runs_on": f"host cores ({cores} spawned processes); rank 0 only",
        "cpu_baseline": {"value": value, "unit": "cell·k-pts/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cell·k-pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_dict(wl, ngpu):
    """The workload's description; identical for both arms (where each arm runs is stated outside it)."""
    walls = {"dirichlet": "Dirichlet walls (Fermi-Dirac beta=1, mu=0)",
             "maxwell": f"Maxwell walls (alpha={wl.get('alpha', 0)}, Fermi-Dirac beta=1, mu=0)",
             "periodic": "periodic"}[wl["bc"]]
    form = "plain FP64" if wl.get("precision", 0) == 0 else "FP32-split (FP32 collision transforms, FP64 rest)"
    return {
        "workload": (f"{wl['name']}: {form}, {wl['N']}x{wl['N']} velocity grid, Nx={wl['Nx']} cells, {walls}, "
                     f"B={tuple(wl['B'])}, dt={wl['dt']}, J=M={wl['J']}, L={wl['L']}, R={wl['R']}, "
                     f"{int(100 * wl['perturb'])}% perturbed synthetic W"),
        "N": wl["N"], "Nx": wl["Nx"], "J": wl["J"], "M": wl["M"], "dt": wl["dt"],
        "bc": wl["bc"], "B": list(wl["B"]), "precision": "f64" if wl.get("precision", 0) == 0 else "f32-split",
        "l2": ("GPU arm: 256 MiB buffer zeroed before every timed step (working set also exceeds L2); "
               "reference arm (host cores): no flush"),
        "parallelism": "single GPU" if ngpu == 1 else f"{ngpu} replicas",
    }


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_sel):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.sel = device_sel

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.sel is not None:
            cmd += ["-i", str(self.sel)]
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_sm_max():
    try:
        return float(json.load(open(MEASURED_PEAKS)).get("sm_max_mhz", 2070.0))
    except Exception:
        return 2070.0


def gpu_uuid(local):
    import torch

    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    import __graft_entry__ as g

    g.build()
    from paper_1408_1782_gb300 import decomp, inputs, qbe

    if args.mode == "peaks":
        return run_peaks(local)
    if args.workload in ("batched_16", "batched_64"):
        return run_batched(args, local, full=args.workload == "batched_64")
    if args.workload == "adjoint_n64":
        return run_adjoint(args, local)
    wl = workload(args.workload, args.precision)
    if args.velocity_n and args.mode in ("collide", "vjp"):
        wl["N"] = args.velocity_n
        wl["name"] += f" at N={args.velocity_n}"
    if args.mode == "collide":
        return run_collide_only(args, wl, local)
    if args.mode == "vjp":
        return run_vjp_only(args, wl, local)
    N, Nx = wl["N"], wl["Nx"]
    prec = wl.get("precision", 0)
    stream = torch.cuda.current_stream()
    s = qbe.Solver(N, Nx, J=wl["J"], M=wl["M"], L=wl["L"], R=wl["R"], device=local, stream=stream,
                   precision=prec)
    if wl["bc"] != "periodic":
        fd = qbe.fd_state(wl["wall"]["beta"], wl["wall"]["mu_up"], wl["wall"]["mu_dn"])
        s.set_boundary(wl["bc"], fd, fd, alpha=wl.get("alpha", 0.0))
    s.set_bfield(inputs.uniform_b(Nx, wl["B"]))
    W0 = inputs.synthetic_w(N, Nx, L=wl["L"], seed=0, perturb=wl["perturb"])
    s.set_state(W0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):                 # the same launches as a timed step, flush included
        flush.zero_()
        s.step(wl["dt"], 1)
    torch.cuda.synchronize()

    clocks = ClockSampler(gpu_uuid(local))
    s.enable_timing(True)
    launches0 = s.launch_count()
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        flush.zero_()
        s.step(wl["dt"], 1)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = s.launch_count() - launches0
    t_ms = decomp.max_over_ranks(e0.elapsed_time(e1))
    groups = {}
    for gname in qbe.KERNEL_GROUPS:
        ms, cnt = s.kernel_time(gname)
        groups[gname] = {"ms": ms, "launches": cnt}
    s.enable_timing(False)

    units_per_step = 2 * Nx * N * N
    value = world * args.steps * units_per_step / (t_ms * 1e-3)

    # end to end through host buffers: pinned host state in, step, state out
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    host = torch.from_numpy(W0).pin_memory()
    host_out = torch.empty_like(host).pin_memory()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_state(host)            # H2D from pinned host memory inside the C call
        s.step(wl["dt"], 1)
        s.get_state(host_out)        # D2H of the step's result (synchronises)
    t_e2e = decomp.max_over_ranks(time.perf_counter() - t0)
    e2e_value = world * e2e_steps * units_per_step / t_e2e
    state_bytes = W0.nbytes

    # roofline of the dominant kernel (I3, Hu-Ying term): FP64 ALU bound
    i3 = groups["i3"]
    avg_i3_s = i3["ms"] * 1e-3 / max(i3["launches"], 1)
    flops_per_launch = Nx * wl["J"] * wl["M"] * i3_flops_per_unit(N)
    achieved = flops_per_launch / avg_i3_s / 1e12
    sm_max = measured_sm_max()
    lanes = FP64_FMA_PER_CLK_PER_SM if prec == 0 else FP32_FMA_PER_CLK_PER_SM
    peak = SM_COUNT * lanes * 2 * sm_max * 1e6 / 1e12
    total_group_ms = sum(v["ms"] for v in groups.values())

    # the streaming kernels (transport, RK/precession): algorithmic bytes and FP64 operations per
    # launch over their live CUDA-event duration, against the measured copy bandwidth and the FP64
    # issue rate (FP64_FMA_PER_CLK_PER_SM lanes per clock per SM): on this part an FP64 stream of a
    # few operations per 8-byte word is bound by the FP64 pipe before HBM.
    hbm_peak = 6778.0
    try:
        hbm_peak = float(json.load(open(MEASURED_PEAKS)).get("hbm_gbs", hbm_peak))
    except Exception:
        pass
    fp64_ops_peak = SM_COUNT * FP64_FMA_PER_CLK_PER_SM * sm_max * 1e6
    nvel = Nx * N * N
    sb = nvel * 4 * 8
    streaming = {}
    # k_advect: per output value 3 differences, 1 subtraction, 2 FMAs; reads and writes the state once.
    # k_rk1 / k_rk2 (one timing group, per-kernel averages): 16 and 20 FP64 operations per velocity;
    # 16 and 20 words of traffic per velocity (k_rk1: W, C in, F0, W1 out; k_rk2: W, F0, C1, W1 in, W out).
    for gname, label, bytes_per_launch, ops_per_launch in (
            ("transport", "k_advect", 2 * sb, 6 * 4 * nvel),
            ("rk", "k_rk1+k_rk2 (per kernel)", (16 + 20) / 2 * 8 * nvel, (16 + 20) / 2 * nvel)):
        ms, cnt = groups[gname]["ms"], groups[gname]["launches"]
        if cnt and ms > 0:
            t_launch = ms / cnt * 1e-3
            gbs = bytes_per_launch / t_launch / 1e9
            streaming[label] = {"bytes_per_launch": bytes_per_launch, "fp64_ops_per_launch": ops_per_launch,
                                "avg_launch_us": 1e6 * t_launch, "GB_s": gbs, "frac_of_hbm": gbs / hbm_peak,
                                "frac_of_fp64_issue": ops_per_launch / t_launch / fp64_ops_peak}

    precision_report = None
    if prec == 1 and rank == 0:
        precision_report = fp32_split_report(wl, W0, local, qbe, torch, np)
    forms = None
    if args.workload == "plain_fp64_n64" and world == 1 and not args.no_forms:
        forms = measure_forms(args, wl, W0, s, t_ms / args.steps, local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ncores = min(16, host_cores())
        times, cores = oracle_sample(wl, ncores, repeats=1)
        cpu = {"value": N * N / times[0], "unit": "cell·k-pts/s", "cores": cores, "kind": "oracle",
               "sample": (f"C[W] of 1 of the {Nx} cells (N={N}, J=M={wl['J']}): the oracle's 60 integral "
                          f"terms on {cores} spawned processes, {times[0]:.1f} s")}

    if rank == 0:
        line = {
            "metric": "C[W] cell·k-pts/s", "value": value, "unit": "cell·k-pts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "steps_per_s": 1e3 * args.steps / t_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == 0 else "f32-split",
            "data": "synthetic (seeded Fermi-Dirac-perturbed W, no dataset)",
            "config": config_dict(wl, world),
            "roofline": {"kernel": s.i3_shape()["name"] + " I3 kernel (Hu-Ying term)", "bound": "alu",
                         "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": (I3_DRAM_BYTES_PER_UNIT[(N, prec)] * Nx * wl["J"] * wl["M"]
                                     if (N, prec) in I3_DRAM_BYTES_PER_UNIT else None),
                         "flops_per_launch": flops_per_launch, "avg_launch_ms": avg_i3_s * 1e3,
                         "peak_source": (f"derived: {SM_COUNT} SMs x {lanes} {'FP64' if prec == 0 else 'FP32'} FMA/clk x 2 "
                                         f"flop x {sm_max:.0f} MHz (bench.py --mode peaks at 2070 MHz: DFMA 1.256, "
                                         f"FFMA 76.8 TFLOP/s)")},
            "kernel_share": {k: round(v["ms"] / total_group_ms, 4) for k, v in groups.items()},
            "streaming_kernels": streaming,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "cell·k-pts/s", "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes, "steps": e2e_steps},
            "gpu_launches": launches,
            "clocks": clk,
        }
        if precision_report is not None:
            line["precision_report"] = precision_report
        if forms is not None:
            line["forms"] = forms
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def measure_forms(args, wl, W0, s64, fp64_ms_per_step, local):
    """The rest of the benchmark metric on the same N = 64, Nx = 128 grid: the FP32-split form of
    this workload (steps/s and C[W] cell*k-pts/s with its error against the plain FP64 GPU form and
    the stored oracle cells) and the adjoint/forward ratio of the differentiation configuration
    (periodic, FP32-split) over a short horizon."""
    import numpy as np
    import torch

    from paper_1408_1782_gb300 import inputs, qbe

    N, Nx = wl["N"], wl["Nx"]
    stream = torch.cuda.current_stream()
    s = qbe.Solver(N, Nx, J=wl["J"], M=wl["M"], L=wl["L"], R=wl["R"], device=local, stream=stream, precision=1)
    fd = qbe.fd_state(wl["wall"]["beta"], wl["wall"]["mu_up"], wl["wall"]["mu_dn"])
    s.set_boundary(wl["bc"], fd, fd, alpha=wl.get("alpha", 0.0))
    s.set_bfield(inputs.uniform_b(Nx, wl["B"]))
    s.set_state(W0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        flush.zero_()
        s.step(wl["dt"], 1)
    torch.cuda.synchronize()
    steps = max(args.steps, 5)
    sampler = ClockSampler(gpu_uuid(local))
    s.enable_timing(True)
    launches0 = s.launch_count()
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        flush.zero_()
        s.step(wl["dt"], 1)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = sampler.stop()
    t_ms = e0.elapsed_time(e1)
    launches = s.launch_count() - launches0
    i3_ms, i3_n = s.kernel_time("i3")
    s.enable_timing(False)
    units = 2 * Nx * N * N
    # end to end: the state in from pinned host memory and out again around each step
    host = torch.from_numpy(W0).pin_memory()
    host_out = torch.empty_like(host).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(steps, args.e2e_steps))
    for _ in range(e2e_steps):
        s.set_state(host)
        s.step(wl["dt"], 1)
        s.get_state(host_out)
    t_e2e = time.perf_counter() - t0
    # error of C[W] at the initial state: every cell against the FP64 GPU form, and the stored
    # oracle cells of this workload
    w = torch.from_numpy(W0).cuda()
    c32 = s.collide(w).cpu().numpy()
    c64 = s64.collide(w).cpu().numpy()
    paper_norm = lambda a, b: float(max(sum(np.abs(a[i, k] - b[i, k]).sum() / np.abs(b[i, k]).sum()
                                            for k in range(4)) for i in range(a.shape[0])))
    err = {"max_rel_vs_fp64_gpu": float(np.abs(c32 - c64).max() / np.abs(c64).max()),
           "paper_norm_vs_fp64_gpu": paper_norm(c32, c64), "cells_compared_with_fp64_gpu": Nx}
    gold = os.path.join(ROOT, "tests", "golden", "plain_fp64_n64_cells.npz")
    if os.path.exists(gold):
        g = np.load(gold)
        cg = c32[g["cells"]]
        err["max_rel_vs_oracle_cells"] = float(np.abs(cg - g["C"]).max() / np.abs(g["C"]).max())
        err["paper_norm_vs_oracle_cells"] = paper_norm(cg, g["C"])
        err["oracle_cells"] = [int(c) for c in g["cells"]]
    err["tolerance_max_rel"] = 5e-6
    err["tolerance_paper_norm"] = 5e-5
    err["within_tolerance"] = bool(err["max_rel_vs_fp64_gpu"] < 5e-6 and err["paper_norm_vs_fp64_gpu"] < 5e-5 and
                                   err.get("max_rel_vs_oracle_cells", 0) < 5e-6 and
                                   err.get("paper_norm_vs_oracle_cells", 0) < 5e-5)
    sm_max = measured_sm_max()
    peak32 = SM_COUNT * FP32_FMA_PER_CLK_PER_SM * 2 * sm_max * 1e6 / 1e12
    avg_i3 = i3_ms * 1e-3 / max(i3_n, 1)
    achieved = Nx * wl["J"] * wl["M"] * i3_flops_per_unit(N) / avg_i3 / 1e12
    fp32 = {
        "form": "FP32-split: collision transforms and products in FP32; input, output, partial-sum reduction, "
                "transport, RK2 and moments in FP64",
        "metric": "C[W] cell·k-pts/s", "value": steps * units / (t_ms * 1e-3), "unit": "cell·k-pts/s",
        "steps": steps, "warmup": args.warmup, "ms_per_step": t_ms / steps, "steps_per_s": 1e3 * steps / t_ms,
        "speedup_vs_fp64_gpu_step": fp64_ms_per_step / (t_ms / steps),
        "error": err,
        "roofline": {"kernel": s.i3_shape()["name"] + " I3 kernel (Hu-Ying term, FP32)", "bound": "alu",
                     "achieved": achieved, "peak": peak32, "unit": "TFLOP/s", "frac": achieved / peak32,
                     "traffic": I3_DRAM_BYTES_PER_UNIT[(64, 1)] * Nx * wl["J"] * wl["M"] if N == 64 else None,
                     "avg_launch_ms": avg_i3 * 1e3,
                     "peak_source": f"derived: {SM_COUNT} SMs x {FP32_FMA_PER_CLK_PER_SM} FP32 FMA/clk x 2 flop x "
                                    f"{sm_max:.0f} MHz"},
        "e2e": {"value": e2e_steps * units / t_e2e, "unit": "cell·k-pts/s", "h2d_bytes_per_step": W0.nbytes,
                "d2h_bytes_per_step": W0.nbytes, "steps": e2e_steps},
        "gpu_launches": launches, "clocks": clk,
    }
    s.close()
    awl = workload("adjoint_n64")
    H, every = args.forms_horizon, 1
    adj = measure_adjoint(awl, local, H, every, steps=2, warmup=1, cpu_baseline=False, clocks=True, tape="full")
    ck = measure_adjoint(awl, local, H, every, steps=2, warmup=1, cpu_baseline=False, clocks=False,
                         tape="checkpoint")
    adj["checkpointed"] = {k: ck[k] for k in ("value", "unit", "forward_ms_per_split_step",
                                               "reverse_ms_per_split_step_both_gradients", "e2e")}
    adj["checkpointed"]["tape_bytes"] = ck["config"]["tape_bytes"]
    adj["note"] = (f"the differentiation configuration (N=64, Nx=128, periodic, B=(0.3,0,0.4), FP32-split) "
                   f"over {H} split steps; value: the forward keeps every intermediate state (full tape, "
                   f"{adj['config']['tape_bytes'] / 1e9:.2f} GB here, {tape_bytes(awl, 200, True) / 1e9:.1f} GB "
                   f"for the 200-step horizon), so the reverse sweep recomputes nothing; 'checkpointed': a "
                   f"checkpoint every step, each step recomputed once by the reverse sweep.  The per-step "
                   f"ratios do not depend on the horizon")
    return {"fp32_split": fp32, "adjoint": adj}


def fp32_split_report(wl, W0, local, qbe, torch, np):
    """FP32-split C[W] against the plain FP64 GPU form on a sample of cells (speed and error), and
    against the stored FP64 oracle cells of this workload when present."""
    N, J, M = wl["N"], wl["J"], wl["M"]
    ncell = min(16, wl["Nx"])
    w = torch.from_numpy(np.ascontiguousarray(W0[:ncell])).cuda()
    out = {}
    res = {}
    for prec in (0, 1):
        s = qbe.Solver(N, ncell, J=J, M=M, L=wl["L"], R=wl["R"], device=local,
                       stream=torch.cuda.current_stream(), precision=prec)
        c = s.collide(w)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.collide(w, c)
        e1.record()
        torch.cuda.synchronize()
        res[prec] = (c.cpu().numpy(), e0.elapsed_time(e1))
        s.close()
    ref, t64 = res[0]
    got, t32 = res[1]
    out["sample_cells"] = ncell
    out["ms_fp64_gpu"] = t64
    out["ms_fp32_split"] = t32
    out["speedup_vs_fp64_gpu"] = t64 / t32
    out["max_rel_err_vs_fp64_gpu"] = float(np.abs(got - ref).max() / np.abs(ref).max())
    out["tolerance_max_rel"] = 5e-6
    gold = os.path.join(ROOT, "tests", "golden",
                        "precision_n128_cells.npz" if N == 128 else "plain_fp64_n64_cells.npz")
    if os.path.exists(gold):
        g = np.load(gold)
        s = qbe.Solver(N, len(g["cells"]), J=J, M=M, L=wl["L"], R=wl["R"], device=local,
                       stream=torch.cuda.current_stream(), precision=1)
        c = s.collide(torch.from_numpy(g["W"]).cuda()).cpu().numpy()
        s.close()
        out["max_rel_err_vs_oracle_cells"] = float(np.abs(c - g["C"]).max() / np.abs(g["C"]).max())
        out["paper_norm_err_vs_oracle_cells"] = float(max(
            sum(np.abs(c[i, k] - g["C"][i, k]).sum() / np.abs(g["C"][i, k]).sum() for k in range(4))
            for i in range(c.shape[0])))
        out["tolerance_paper_norm"] = 5e-5
    return out


def run_batched(args, local, full=False):
    """Independent simulations stepped with one CUDA graph launch per split step: 16 drawn with
    N in {32, 48, 64}, Nx in [16, 64] (batched_16), or the full mix of 64 with N in
    {32, 48, 64, 96, 128}, Nx in [16, 256] (batched_64)."""
    import numpy as np
    import torch

    import __graft_entry__ as g

    g.build()
    from paper_1408_1782_gb300 import inputs, qbe

    rng = np.random.default_rng(0)
    stream = torch.cuda.current_stream()
    sims, desc = [], []
    units = 0
    nsims = 64 if full else 16
    grids = [32, 48, 64, 96, 128] if full else [32, 48, 64]
    nx_max = 257 if full else 65
    for i in range(nsims):
        N = int(rng.choice(grids))
        Nx = int(rng.integers(16, nx_max))
        bc = str(rng.choice(["periodic", "dirichlet", "maxwell"]))
        B = rng.normal(size=3)
        B *= rng.uniform(0, 1) / np.linalg.norm(B)
        s = qbe.Solver(N, Nx, J=32, M=32, device=local, stream=stream, precision=1)
        if bc != "periodic":
            fd = qbe.fd_state(1.0, 0.0, 0.0)
            s.set_boundary(bc, fd, fd, alpha=0.5)
        s.set_bfield(inputs.uniform_b(Nx, B))
        s.set_state(inputs.synthetic_w(N, Nx, seed=100 + i, perturb=0.05))
        sims.append(s)
        desc.append(f"{N}/{Nx}/{bc[0]}")
        units += 2 * Nx * N * N
    b = qbe.Batch(sims, stream=stream)
    dt = 0.005

    def timed_steps():
        b.step(dt, args.warmup)            # the first call captures the graph
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(dt, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    states = [s.get_state() for s in sims]
    untuned_ms = None
    if args.compare_untuned:
        untuned_ms = timed_steps() / args.steps
        for s, W in zip(sims, states):
            s.set_state(W)
    t0 = time.perf_counter()
    shapes = b.autotune()
    tune_s = time.perf_counter() - t0
    groups = {}
    for s, (gg, mm, ms) in zip(sims, shapes):
        sh = s.i3_shape()
        groups.setdefault((s.N, s.precision), {"N": s.N, "variant": sh["name"], "grid": gg, "m_chunks": mm,
                                               "predicted_i3_ms": round(ms, 3), "sims": 0})["sims"] += 1
    t_ms = timed_steps()
    line = {"workload": "batched_64" if full else "batched_16", "metric": "C[W] cell·k-pts/s",
            "value": units * args.steps / (t_ms * 1e-3),
            "unit": "cell·k-pts/s", "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "untuned_ms_per_step": untuned_ms, "autotune_s": round(tune_s, 2),
            "dtype": "f32-split", "graph_launches_per_step": 1,
            "sims": desc, "tuned_i3_shapes": list(groups.values()),
            "note": ("the batching configuration: 64 simulations, N from {32,48,64,96,128}, Nx from [16,256], "
                     "mixed walls, random |B| <= 1; one I3 work-queue launch per padded size, its launch shape "
                     "chosen by qbe_batch_autotune" if full else
                     "16 simulations drawn from the batching configuration's distributions with N in {32,48,64} "
                     "and Nx in [16,64]; --workload batched_64 runs the full 64-simulation mix")}
    print(json.dumps(line), flush=True)
    b.close()
    for s in sims:
        s.close()
    return 0


def run_peaks(local):
    """Arithmetic issue rates of the GPU (qbe_arith_issue_rates), per second and per clock per SM at
    the SM clock sampled while they ran: the measurement behind the derived "alu" peaks."""
    import torch

    from paper_1408_1782_gb300 import qbe

    stream = torch.cuda.current_stream()
    qbe.arith_issue_rates(local, stream)          # warm-up (clocks, module load)
    sampler = ClockSampler(gpu_uuid(local))
    sampler.start()
    runs = [qbe.arith_issue_rates(local, stream) for _ in range(20)]   # about 1.5 s for the clock samples
    clk = sampler.stop()
    rates = {k: statistics.median(r[k] for r in runs) for k in runs[0]}
    mhz = clk.get("sm_mhz") or measured_sm_max()
    line = {"mode": "peaks", "lane_ops_per_s": rates,
            "per_clk_per_sm": {k: v / (SM_COUNT * mhz * 1e6) for k, v in rates.items()},
            "fp64_fma_tflops": 2 * rates["dfma"] / 1e12, "fp32_fma_tflops": 2 * rates["ffma"] / 1e12,
            "derived_peaks_tflops": {"fp64": SM_COUNT * FP64_FMA_PER_CLK_PER_SM * 2 * measured_sm_max() / 1e6,
                                     "fp32": SM_COUNT * FP32_FMA_PER_CLK_PER_SM * 2 * measured_sm_max() / 1e6},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_collide_only(args, wl, local):
    """C[W] evaluations of the first `cells` cells of the workload's initial state."""
    import torch

    from paper_1408_1782_gb300 import inputs, qbe

    N = wl["N"]
    cells = args.cells or wl["Nx"]
    stream = torch.cuda.current_stream()
    s = qbe.Solver(N, cells, J=wl["J"], M=wl["M"], L=wl["L"], R=wl["R"], device=local, stream=stream,
                   precision=wl.get("precision", 0))
    W = inputs.synthetic_w(N, wl["Nx"], L=wl["L"], seed=0, perturb=wl["perturb"])[:cells]
    w = torch.from_numpy(W.copy()).cuda()
    c = torch.empty_like(w)
    tuned_ms = None
    if args.autotune:
        s.set_state(W.copy())
        tuned_ms = s.autotune()
    if args.i3_variant >= 0:
        s.set_i3_shape(variant=args.i3_variant)
    for _ in range(args.warmup):
        s.collide(w, c)
    torch.cuda.synchronize()
    s.enable_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        s.collide(w, c)
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1)
    i3_ms, i3_n = s.kernel_time("i3")
    flops = cells * wl["J"] * wl["M"] * i3_flops_per_unit(N)
    line = {"mode": "collide", "metric": "C[W] cell·k-pts/s", "value": args.steps * cells * N * N / (t_ms * 1e-3),
            "unit": "cell·k-pts/s", "cells": cells, "steps": args.steps, "warmup": args.warmup,
            "ms_per_eval": t_ms / args.steps, "i3_ms_per_launch": i3_ms / max(i3_n, 1),
            "i3_tflops": flops / (i3_ms / max(i3_n, 1) * 1e-3) / 1e12,
            "dtype": "f64" if wl.get("precision", 0) == 0 else "f32-split", "workload": wl["name"],
            "i3_shape": s.i3_shape(), "autotune_predicted_ms": tuned_ms}
    print(json.dumps(line), flush=True)
    s.close()
    return 0


def i3_vjp_flops_per_unit(N, K=1):
    """Algorithmic FLOPs of one (cell, j, m) unit of the I3 transpose kernel carrying K cotangents,
    same convention as i3_flops_per_unit.  Per cotangent: 72 real 2-D transforms (4 for the two
    shifts, 64 for the 16 convolutions of complex pairs, 4 for the two forward transforms of the
    shifted-back sums) at 2.5 P log2 P each, plus 228 P pointwise flops (shift phases, 16 scalings,
    16 psi' products, the three pointwise sums per component, the conjugate phases and spectral
    accumulation).  K cotangents at one state share the shifts and the 8 convolutions of the state
    (36 real transforms), so the launch does 36 + 36 K of them."""
    P = (2 * N) ** 2
    return 2.5 * P * math.log2(P) * (36.0 + 36.0 * K) + 228.0 * P * K


def vjp_cotangent_group(prec, N, ncot):
    """Cotangents one collision product carries in the library (the FP32-split form on padded grids
    up to 128 points takes one at a time, the staged forms up to four)."""
    return 1 if (prec == 1 and 2 * N <= 128) else min(ncot, 4)


def run_adjoint(args, local):
    """Gradient of the final-time spin polarisation P_z and energy flux Phi_E with respect to the
    initial state W_0 and the field B: forward sweep (qbe_step_checkpointed over the horizon) and
    reverse sweep (qbe_observables_vjp + qbe_step_vjp).  One timed step = one gradient of both
    observables (one forward sweep, one reverse sweep carrying both cotangents)."""
    wl = workload("adjoint_n64", args.precision)
    H = args.horizon or wl["checkpoint_every"]
    every = min(wl["checkpoint_every"], H)
    line = measure_adjoint(wl, local, H, every, args.steps, args.warmup,
                           cpu_baseline=not args.no_cpu_baseline, clocks=True, tape=args.tape)
    line.update({"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "scaling": "weak", "vs_baseline": None,
                 "data": "synthetic (seeded Fermi-Dirac-perturbed W, no dataset)"})
    print(json.dumps(line), flush=True)
    return 0


def tape_bytes(wl, H, full):
    """Device memory of the forward's tape: every intermediate state of the H steps (full), or one
    checkpoint segment's, which the reverse sweep recomputes (2 s + 2 states per step, s the transport
    substeps of a half step, as the library counts them)."""
    import math

    s = max(1, math.ceil(0.5 * wl["dt"] * wl["L"] * wl["Nx"] - 1e-12))
    return (H if full else 1) * (2 * s + 2) * wl["Nx"] * 4 * wl["N"] ** 2 * 8


def measure_adjoint(wl, local, H, every, steps, warmup, cpu_baseline=True, clocks=True, tape="full"):
    """Time `steps` gradients of (P_z, Phi_E) after H split steps of the workload `wl`; returns the
    adjoint/forward ratio with its roofline, e2e and kernel times.  tape="full": the forward keeps every
    intermediate state (qbe_step_taped) and the reverse sweep recomputes nothing; "checkpoint": a
    checkpoint every `every` steps, each segment recomputed once by the reverse sweep."""
    import numpy as np
    import torch

    from paper_1408_1782_gb300 import inputs, qbe

    N, Nx, prec = wl["N"], wl["Nx"], wl.get("precision", 0)
    stream = torch.cuda.current_stream()
    s = qbe.Solver(N, Nx, J=wl["J"], M=wl["M"], L=wl["L"], R=wl["R"], device=local, stream=stream,
                   precision=prec)
    if wl["bc"] != "periodic":
        fd = qbe.fd_state(wl["wall"]["beta"], wl["wall"]["mu_up"], wl["wall"]["mu_dn"])
        s.set_boundary(wl["bc"], fd, fd, alpha=wl.get("alpha", 0.0))
    B = torch.from_numpy(inputs.uniform_b(Nx, wl["B"])).cuda()
    W0 = torch.from_numpy(inputs.synthetic_w(N, Nx, L=wl["L"], seed=0, perturb=wl["perturb"])).cuda()
    lams = torch.empty((2,) + tuple(W0.shape), dtype=torch.float64, device="cuda")
    lam0s = torch.empty_like(lams)
    gBs = torch.empty((2,) + tuple(B.shape), dtype=torch.float64, device="cuda")
    obs = torch.empty(2, dtype=torch.float64, device="cuda")
    seeds = [torch.tensor([1.0, 0.0], dtype=torch.float64, device="cuda"),
             torch.tensor([0.0, 1.0], dtype=torch.float64, device="cuda")]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def record():
        if tape == "full":
            s.step_taped(wl["dt"], H)
        else:
            s.step_checkpointed(wl["dt"], H, every)

    def gradient(events=None):
        s.set_state(W0)
        s.set_bfield(B)
        if events:
            events[0].record(stream)
        record()
        s.observables(None, out=obs)
        if events:
            events[1].record(stream)
        for k, g in enumerate(seeds):
            s.observables_vjp(g, out=lams[k])
        s.step_vjp_many(lams, out=lam0s, grad_B=gBs)      # both gradients in one reverse sweep
        if events:
            events[2].record(stream)

    for _ in range(warmup):
        flush.zero_()
        gradient()
    torch.cuda.synchronize()
    vjp_variant = s.vjp_i3_variant()[0]
    sampler = ClockSampler(gpu_uuid(local)) if clocks else None
    s.enable_timing(True)
    launches0 = s.launch_count()
    if sampler:
        sampler.start()
    fwd, rev = 0.0, 0.0
    for _ in range(steps):
        flush.zero_()
        e = [ev(), ev(), ev()]
        gradient(e)
        torch.cuda.synchronize()
        fwd += e[0].elapsed_time(e[1])
        rev += e[1].elapsed_time(e[2])
    clk = sampler.stop() if sampler else None
    launches = s.launch_count() - launches0
    vi3_ms, vi3_n = s.kernel_time("vjp_i3")
    groups = {gname: s.kernel_time(gname)[0] for gname in qbe.KERNEL_GROUPS}
    s.enable_timing(False)
    # reverse work per observable gradient (two gradients share one sweep) over the forward sweep
    ratio = (rev / 2.0) / fwd
    avg_vi3 = vi3_ms * 1e-3 / max(vi3_n, 1)
    kgrp = vjp_cotangent_group(prec, N, 2)            # the sweep carries two cotangents
    flops = Nx * wl["J"] * wl["M"] * i3_vjp_flops_per_unit(N, kgrp)
    sm_max = measured_sm_max()
    lanes = FP64_FMA_PER_CLK_PER_SM if prec == 0 else FP32_FMA_PER_CLK_PER_SM
    peak = SM_COUNT * lanes * 2 * sm_max * 1e6 / 1e12
    achieved = flops / avg_vi3 / 1e12

    # end to end through host buffers: state and field in from pinned host memory, gradients out
    hW = W0.cpu().pin_memory()
    hB = B.cpu().pin_memory()
    hl = torch.empty_like(hW).pin_memory()
    hl0 = torch.empty_like(hW).pin_memory()
    hgB = torch.empty_like(hB).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_state(hW)
    s.set_bfield(hB)
    record()
    obs_host = s.observables()            # D2H of the observables (synchronises)
    t1 = time.perf_counter()
    s.observables_vjp(np.array([1.0, 0.0]), out=hl)
    s.step_vjp(hl, out=hl0, grad_B=hgB)
    t2 = time.perf_counter()
    cpu = adjoint_cpu_baseline(wl) if cpu_baseline else None
    conf = config_dict(wl, 1)
    vjp_kernel = "k_i3_vjp"                            # the staged form (FP64; FP32 above 128 points)
    if prec == 1 and 2 * N <= 128:
        vjp_kernel = "k_i3_vjp_wl" if (2 * N == 128 and kgrp == 1 and vjp_variant == 0) else "k_i3_vjp_smem"
    how = ("full tape: every intermediate state kept" if tape == "full"
           else f"checkpoint every {every}, segments recomputed")
    conf.update({"horizon_steps": H, "tape": tape, "checkpoint_every": every if tape != "full" else None,
                 "tape_bytes": tape_bytes(wl, H, tape == "full"),
                 "workload": conf["workload"] + f"; gradient of P_z and Phi_E after {H} split steps "
                                                f"({how}) w.r.t. W_0 and B"})
    line = {
        "metric": "adjoint/forward time ratio", "value": ratio,
        "unit": "reverse s per observable gradient (P_z and Phi_E in one sweep) / forward sweep s",
        "ms_per_step": (fwd + rev) / steps, "higher_is_better": False,
        "dtype": "f64" if prec == 0 else "f32-split", "config": conf,
        "forward_ms_per_split_step": fwd / steps / H,
        "reverse_ms_per_split_step_both_gradients": rev / steps / H,
        "gradients_per_s": 2e3 * steps / (fwd + rev),
        "observables": obs.cpu().tolist(),
        "roofline": {"kernel": f"{vjp_kernel} (transpose of the Hu-Ying I3 term)", "bound": "alu",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": (I3_VJP_DRAM_BYTES_PER_UNIT[(N, prec)] * Nx * wl["J"] * wl["M"]
                                 if (N, prec) in I3_VJP_DRAM_BYTES_PER_UNIT and kgrp == 1 else None),
                     "flops_per_launch": flops, "avg_launch_ms": avg_vi3 * 1e3,
                     "peak_source": (f"derived: {SM_COUNT} SMs x {lanes} {'FP64' if prec == 0 else 'FP32'} "
                                     f"FMA/clk x 2 flop x {sm_max:.0f} MHz")},
        "kernel_ms": {k: round(v, 2) for k, v in groups.items()},
        "cpu_baseline": cpu,
        "e2e": {"value": (t2 - t1) / (t1 - t0), "unit": "reverse sweep s / forward sweep s (one observable)",
                "h2d_bytes_per_step": hW.numel() * 8 + hB.numel() * 8 + 16,
                "d2h_bytes_per_step": obs_host.nbytes + hl.numel() * 8 * 2 + hgB.numel() * 8,
                "note": "one observable's gradient; forward sweep incl. H2D of W_0 and B, reverse incl. D2H"},
        "gpu_launches": launches,
    }
    if clk is not None:
        line["clocks"] = clk
    s.close()
    return line


def adjoint_cpu_baseline(wl):
    """The oracle's derivative of C[W] along one direction for one cell (forward mode: four C[W]
    evaluations of the five-point difference), on up to 16 spawned processes."""
    import multiprocessing as mp

    from oracle import qbe_oracle as O
    from oracle import tangent as T
    from paper_1408_1782_gb300 import inputs

    p = O.Params(N=wl["N"], L=wl["L"], R=wl["R"], J=wl["J"], M=wl["M"])
    W = inputs.synthetic_w(wl["N"], 1, L=wl["L"], seed=0, perturb=wl["perturb"])
    dW = inputs.random_field(W.shape, seed=1, scale=0.05)
    ncores = min(16, host_cores())
    with mp.get_context("spawn").Pool(ncores) as pool:
        t = time.perf_counter()
        T.collision_jvp(W, dW, p, mapper=lambda f, it: pool.map(f, list(it), chunksize=1))
        dt = time.perf_counter() - t
    return {"value": wl["N"] ** 2 / dt, "unit": "cell·k-pts/s of dC/dW products", "cores": ncores,
            "kind": "oracle",
            "sample": f"one directional derivative of C[W] for 1 cell (N={wl['N']}, J=M={wl['J']}), {dt:.1f} s"}


def run_vjp_only(args, wl, local):
    """Collision VJPs (dC/dW)^T lam of the first `cells` cells of the workload's initial state."""
    import numpy as np
    import torch

    from paper_1408_1782_gb300 import inputs, qbe

    N = wl["N"]
    cells = args.cells or wl["Nx"]
    stream = torch.cuda.current_stream()
    s = qbe.Solver(N, cells, J=wl["J"], M=wl["M"], L=wl["L"], R=wl["R"], device=local, stream=stream,
                   precision=wl.get("precision", 0))
    W = inputs.synthetic_w(N, wl["Nx"], L=wl["L"], seed=0, perturb=wl["perturb"])[:cells]
    w = torch.from_numpy(W.copy()).cuda()
    K = max(1, args.cotangents)
    s.set_vjp_i3_variant(args.vjp_i3_variant)
    lam = torch.from_numpy(np.stack([inputs.random_field(W.shape, seed=1 + k) for k in range(K)])).cuda()
    g = torch.empty_like(lam)

    def product():
        if K == 1:
            s.collide_vjp(w, lam[0], out=g[0])
        else:
            s.collide_vjp_many(w, lam, out=g)

    for _ in range(args.warmup):
        product()
    torch.cuda.synchronize()
    s.enable_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        product()
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1)
    v_ms, v_n = s.kernel_time("vjp_i3")
    # one I3 transpose launch carries a group of the K products; algorithmic work of such a launch
    kgrp = vjp_cotangent_group(wl.get("precision", 0), N, K)
    flops = cells * wl["J"] * wl["M"] * i3_vjp_flops_per_unit(N, kgrp)
    line = {"mode": "vjp", "metric": "dC/dW^T products, cell·k-pts/s",
            "value": K * args.steps * cells * N * N / (t_ms * 1e-3),
            "unit": "cell·k-pts/s", "cells": cells, "cotangents": K, "steps": args.steps, "warmup": args.warmup,
            "ms_per_product": t_ms / args.steps / K, "vjp_i3_ms_per_launch": v_ms / max(v_n, 1),
            "cotangents_per_launch": kgrp, "vjp_i3_tflops": flops / (v_ms / max(v_n, 1) * 1e-3) / 1e12,
            "vjp_i3_variant": s.vjp_i3_variant()[0],
            "dtype": "f64" if wl.get("precision", 0) == 0 else "f32-split", "workload": wl["name"]}
    print(json.dumps(line), flush=True)
    s.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="default workload: skip the FP32-split and adjoint measurements of the same grid")
    ap.add_argument("--forms-horizon", type=int, default=2,
                    help="split steps of the adjoint measurement inside the default line")
    ap.add_argument("--mode", choices=["step", "collide", "vjp", "peaks"], default="step")
    ap.add_argument("--workload", choices=["plain_fp64_n64", "precision_n128", "batched_16", "batched_64",
                                           "adjoint_n64"],
                    default="plain_fp64_n64")
    ap.add_argument("--horizon", type=int, default=0,
                    help="adjoint_n64: split steps per gradient (default: one checkpoint segment, 20)")
    ap.add_argument("--tape", choices=["full", "checkpoint"], default="full",
                    help="adjoint_n64: keep every intermediate state of the forward (full) or recompute "
                         "each checkpoint segment in the reverse sweep (checkpoint)")
    ap.add_argument("--precision", type=int, choices=[0, 1], default=None)
    ap.add_argument("--cells", type=int, default=0)
    ap.add_argument("--velocity-n", type=int, default=0,
                    help="--mode collide / vjp: velocity grid N instead of the workload's (other padded sizes)")
    ap.add_argument("--i3-variant", type=int, default=-1,
                    help="--mode collide: I3 launch variant (qbe_set_i3_shape); default: the library's")
    ap.add_argument("--autotune", action="store_true", help="--mode collide: run qbe_autotune first")
    ap.add_argument("--vjp-i3-variant", type=int, default=-1,
                    help="--mode vjp: I3 transpose kernel variant (qbe_set_vjp_i3_variant); default: the library's")
    ap.add_argument("--compare-untuned", action="store_true",
                    help="batched workloads: also time the steps with the default launch shapes first")
    ap.add_argument("--cotangents", type=int, default=1,
                    help="--mode vjp: products per call at the same state (shared transforms, up to 4 per group)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
