#!/usr/bin/env python3
"""Benchmark of the GB300 MLMC hot path for the 2-D Dean--Kawasaki equation.

Workload (default ``mlmc16_256``): unit torus, levels 16^2..256^2 (h_l =
1/16..1/256), tau_l ~ 0.1 h_l^2, T = 0.02, N = 1e5, rho0 = 1 + 0.5 sin sin,
phi = cos(2 pi x1), NN-coupled levels, RMSE target eps = 1e-3 relative.

One *step* is one pass of the whole hot path over the workload's MLMC batch:
for every level l, M_l coupled samples (Philox normals, fused fine/coarse
stepping, observables, P, FP64 moment sums; the per-level counts M_l are the
allocation Algorithm 1 reaches for eps = 1e-3), then the estimator and its
variance from the sums (Eq. MLMCEstimator).  ``value`` is coupled
sample-steps per second (sum over levels of M_l x fine steps, per second),
inputs resident on the device; ``e2e`` is the same through the public C-ABI
with host buffers (init uploads the level tables from pinned memory, host
sums are read back per level).  Also reported: the wall time of a full
adaptive Algorithm 1 run to eps and the plain single-level MC time to the
same eps on the finest level reached (sample count 2 Var[P_L] / eps^2 times
the measured MC time per sample).

Under torchrun every rank runs the same batch under its own seed (independent
samples, no collective on the data path): weak scaling.
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

METRIC = "MLMC wall time to RMSE ε vs plain MC (1 GB300); coupled sample-steps/s; HBM GB/s"
UNIT = "coupled sample-steps/s"
# XU-pipe (MUFU) operations the method needs per fine cell-step: Box--Muller
# for the two normals (log, sqrt, sin, cos) and sqrt([rho]^+); per coarse
# cell-step sqrt([rho]^+) only (coarse normals are sums of fine ones).
XU_OPS_FINE = 5.0
XU_OPS_COARSE = 1.0
XU_PER_CLK_PER_SM = 16
SMS = 152
SM_MAX_MHZ = 2070.0
# DRAM bytes of one full-size launch of the dominant kernel (read + write; the
# state never leaves registers, so this is the initial-state, mean-field and
# observable tables), from the one-pass ncu capture of the level kernels of
#   python bench.py --steps 1 --warmup 3 --no-cpu-baseline --no-surrogate --no-adaptive
#       --no-e2e --no-streamed --split-fraction 0.08
# (mean of its 4 launches of 879 samples).  Reported only while the kernel
# sources hash to the value recorded with the capture.
LEVEL_KERNEL_TRAFFIC = {"kernel": "level_kernel n=256 C=4 R=2 cluster=8 coupled=True",
                        "bytes_per_launch": 2.176e6, "sources_sha256_16": "bf4df8416557e594"}
# Thread instructions per fine cell-step of the dominant kernel, from the ncu
# --set full capture of the 256^2 coupled level kernel (smsp__inst_executed x
# 32 / fine cell-steps); valid under the same source hash.  The kernel is
# bound by instruction issue (4 warp instructions per clock per SM).
LEVEL_KERNEL_INSTR_PER_CELL_STEP = 59.0
KERNEL_SOURCES = ("dk_kernels.cu", "dk_device.cuh")   # the level kernel and its device functions


# Theta-scheme kernel (implicit diffusion weight b0 > 0): thread instructions
# per fine cell-step (coupled, coarse work included) of the 64^2 coupled
# launch at b0 = 1/2, tau/h^2 = 0.85 (14 Chebyshev steps per solve), from its
# ncu --set full capture (smsp__inst_executed x 32 / fine cell-steps); valid
# under the recorded hash of its sources.  Bound by instruction issue.
THETA_KERNEL_INSTR = {"kernel": "theta_kernel n=64 coupled=True b0=0.5 chebyshev_steps=14",
                      "instructions_per_fine_cell_step": 580.6, "sources_sha256_16": "5f4fec27e80df0df"}
THETA_SOURCES = ("dk_theta.cu", "dk_device.cuh")
# Fourier-coupled kernel: thread instructions per cell-step (fine and coarse
# cell-steps) of the 54^2 coupled launch, from its ncu --set full capture;
# valid under the recorded hash of its sources.
FOURIER_KERNEL_INSTR = {"kernel": "fourier_kernel n=54 coupled=True",
                        "instructions_per_cell_step": 94.6, "sources_sha256_16": "5eb2d85d130ecf3e"}
FOURIER_SOURCES = ("dk_fourier.cu", "dk_device.cuh")


def kernel_sources_hash(files=KERNEL_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2311_08872_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# Streamed-state stencil: algorithmic bytes per coupled fine cell-step (4 B read
# + 4 B write of the fine state; the coarse state's 8 B every 4th step on a
# quarter of the cells = 0.5 B); the normals are generated in registers.
STREAM_BYTES_PER_FINE_CELL_STEP = 8.5


def measured_peaks():
    """(HBM GB/s, source) from the measured peaks, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def closed_form_EP_cos1(n, tau, M):
    """Martingale-lemma value of E[P] for phi = cos(2 pi x1) on the unit torus
    when rho stays positive (a lower bound otherwise): (tau/2) (sin(2 pi h)/h)^2
    (1 - g^2M) / (1 - g^2), g = 1 - 2 (tau/h^2) sin^2(pi h)."""
    h = 1.0 / n
    g = 1.0 - 2.0 * (tau / (h * h)) * math.sin(math.pi * h) ** 2
    return 0.5 * tau * (math.sin(2 * math.pi * h) / h) ** 2 * (1.0 - g ** (2 * M)) / (1.0 - g * g)


def streamed_stencil(stream):
    """One wave of samples in flight of the 512^2 level of the low-density
    workload on the streamed-state kernels (CUDA events on the launching
    stream; fine-step variant picked by the autotuner)."""
    import torch
    from paper_2311_08872_gb300 import mlmc_dk, workloads
    wl = workloads.get("lowdens32_512")
    level = wl.L_max
    with mlmc_dk.Context.from_workload(wl, stream=stream.cuda_stream) as c:
        c.tune(1)
        info = c.level_info(level)
        S = info.in_flight
        sums = torch.zeros(mlmc_dk.sums_len(c.n_quant), dtype=torch.float64, device="cuda")
        c.run_level_dev(level, 0, 0, 1, 9, sums.data_ptr(), 0, stream.cuda_stream)      # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        c.run_level_dev(level, 0, 1, S, 9, sums.data_ptr(), 0, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
    fine = S * info.n ** 2 * info.M
    peak, src = measured_peaks()
    gbs = fine * STREAM_BYTES_PER_FINE_CELL_STEP / sec / 1e9
    return {"workload": wl.name, "level": level, "n": info.n, "fine_steps": info.M, "samples": S,
            "tile_rows": info.tile_rows, "s": sec, "cell_steps_per_s": S * info.cost / sec,
            "fine_cell_steps_per_s": fine / sec, "algorithmic_bytes_per_fine_cell_step": STREAM_BYTES_PER_FINE_CELL_STEP,
            "achieved_GBps": gbs, "hbm_peak_GBps": peak, "peak_source": src, "frac_of_hbm": gbs / peak,
            "bound": "alu (instruction issue): the working set stays in L2, DRAM traffic is the cold start only"}


def theta_scheme(stream):
    """The theta-scheme kernel on the finest level of the Crank--Nicolson
    workload (64^2 coupled with 32^2, b0 = 1/2, tau/h^2 = 0.85): 32 waves of one
    sample per SM, CUDA events on the launching stream, against the
    instruction-issue roofline."""
    import torch
    from paper_2311_08872_gb300 import mlmc_dk, workloads
    wl = workloads.get("theta16_64")
    level = wl.L_max
    count = 32 * SMS
    with mlmc_dk.Context.from_workload(wl, stream=stream.cuda_stream) as c:
        info = c.level_info(level)
        sums = torch.zeros(mlmc_dk.sums_len(c.n_quant), dtype=torch.float64, device="cuda")
        c.run_level_dev(level, 0, 0, count, 11, sums.data_ptr(), 0, stream.cuda_stream)      # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        c.run_level_dev(level, 0, count, count, 11, sums.data_ptr(), 0, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
    fine = count * info.n ** 2 * info.M
    out = {"workload": wl.name, "level": level, "n": info.n, "fine_steps": info.M, "b0": info.theta_b0,
           "tau_over_h2": info.tau / info.h ** 2, "chebyshev_steps": info.cheb_steps, "samples": count, "s": sec,
           "cell_steps_per_s": count * info.cost / sec, "fine_cell_steps_per_s": fine / sec,
           "coupled_sample_steps_per_s": count * info.M / sec, "bound": "alu (instruction issue)"}
    if kernel_sources_hash(THETA_SOURCES) == THETA_KERNEL_INSTR["sources_sha256_16"]:
        ipc = THETA_KERNEL_INSTR["instructions_per_fine_cell_step"]
        warp_inst = fine * ipc / 32.0 / sec
        peak = 4.0 * SMS * SM_MAX_MHZ * 1e6
        out["issue"] = {"instructions_per_fine_cell_step": ipc, "achieved_warp_inst_per_s": warp_inst,
                        "peak_warp_inst_per_s": peak, "frac": warp_inst / peak}
    return out


def fourier_coupling(stream):
    """The Fourier-coupled kernel on the finest level of fourier6_54 (54^2
    coupled with 18^2, ratio 3): 32 waves of one sample per SM, CUDA events."""
    import torch
    from paper_2311_08872_gb300 import mlmc_dk, workloads
    wl = workloads.get("fourier6_54")
    level = wl.L_max
    count = 32 * SMS
    with mlmc_dk.Context.from_workload(wl, stream=stream.cuda_stream) as c:
        info = c.level_info(level)
        sums = torch.zeros(mlmc_dk.sums_len(c.n_quant), dtype=torch.float64, device="cuda")
        c.run_level_dev(level, 0, 0, count, 13, sums.data_ptr(), 0, stream.cuda_stream)      # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        c.run_level_dev(level, 0, count, count, 13, sums.data_ptr(), 0, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
    out = {"workload": wl.name, "level": level, "n": info.n, "coarse_n": info.n // 3, "fine_steps": info.M,
           "samples": count, "s": sec, "cell_steps_per_s": count * info.cost / sec,
           "coupled_sample_steps_per_s": count * info.M / sec,
           "bound": "alu (instruction issue; shared-memory queue stalls lead)"}
    if kernel_sources_hash(FOURIER_SOURCES) == FOURIER_KERNEL_INSTR["sources_sha256_16"]:
        ipc = FOURIER_KERNEL_INSTR["instructions_per_cell_step"]
        warp_inst = count * info.cost * ipc / 32.0 / sec
        peak = 4.0 * SMS * SM_MAX_MHZ * 1e6
        out["issue"] = {"instructions_per_cell_step": ipc, "achieved_warp_inst_per_s": warp_inst,
                        "peak_warp_inst_per_s": peak, "frac": warp_inst / peak}
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="mlmc16_256")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-streamed", action="store_true", help="skip the streamed-state stencil timing")
    ap.add_argument("--no-theta", action="store_true", help="skip the theta-scheme kernel timing")
    ap.add_argument("--no-fourier", action="store_true", help="skip the Fourier-coupled kernel timing")
    ap.add_argument("--split-fraction", type=float, default=None,
                    help="fixed batch split of the finest cluster level (default: autotuned)")
    ap.add_argument("--no-adaptive", action="store_true", help="skip the Algorithm 1 / plain MC timing")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned level below 0")
    ap.add_argument("--adaptive-eps", type=float, default=1e-2,
                    help="relative eps of the fully measured Algorithm 1 run (0: the workload's)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def level_costs(wl):
    import oracle
    lv = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu, wl.M0)
    fine = [l.n * l.n * l.M for l in lv]
    coarse = [0.0] + [lv[l - 1].n ** 2 * lv[l - 1].M for l in range(1, len(lv))]
    return lv, fine, coarse


def batch_units(wl, alloc):
    lv, fine, coarse = level_costs(wl)
    sample_steps = sum(m * lv[l].M for l, m in enumerate(alloc))
    cell_steps = sum(m * (fine[l] + coarse[l]) for l, m in enumerate(alloc))
    return sample_steps, cell_steps


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle leg
def _oracle_task(args):
    (wl, level, sample) = args
    import oracle
    lv = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu, wl.M0)
    ol = oracle.level_inputs(wl.length, lv, wl.N, wl.rho0_all(), wl.phi_all(), level, level > 0)
    t = time.perf_counter()
    ol.sample(wl.seed, sample, level > 0)
    return level, time.perf_counter() - t


def oracle_rate(wl, alloc, budget_s, cores=None):
    """The FP64 oracle, as it stands, on the host cores: per-level single-core
    seconds per coupled sample measured on a bounded sample (levels with a
    sample of at most ~budget/4 core-seconds), extrapolated by cell-steps to
    the others, then the batch's sample-steps over the batch's CPU time on
    `cores` cores."""
    import multiprocessing as mp
    cores = cores or min(os.cpu_count() or 1, 16)
    lv, fine, coarse = level_costs(wl)
    per_cell = 1.0 / 15e6     # first guess, refined by the measurement below
    tasks = []
    for l in range(len(alloc)):
        est = (fine[l] + coarse[l]) * per_cell
        if est > budget_s * cores / 4:
            continue
        k = max(1, min(64, int(budget_s * cores / (4 * max(est, 1e-6) * len(alloc)))))
        tasks += [(wl, l, 1000 + i) for i in range(k)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_task, tasks, chunksize=1)
    wall = time.perf_counter() - t0
    per_level = {}
    for l, dt in res:
        per_level.setdefault(l, []).append(dt)
    t = {l: statistics.mean(v) for l, v in per_level.items()}
    top = max(t)
    cell_rate = (fine[top] + coarse[top]) / t[top]
    secs = []
    for l, m in enumerate(alloc):
        secs.append(m * (t[l] if l in t else (fine[l] + coarse[l]) / cell_rate))
    sample_steps, cell_steps = batch_units(wl, alloc)
    cpu_time = sum(secs) / cores
    sample = (f"{len(tasks)} coupled samples of levels {sorted(t)} in {wall:.1f} s wall on {cores} processes; "
              f"levels {[l for l in range(len(alloc)) if l not in t]} extrapolated by cell-steps from level {top}")
    return {"value": sample_steps / cpu_time, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": sample, "cell_steps_per_s": cell_steps / cpu_time,
            "cell_steps_per_s_per_core": cell_steps / cpu_time / cores,
            "batch_cpu_s": cpu_time, "wall_s": wall}


# --------------------------------------------------------------- our arm
def run_ours(args, wl, rank, world, local_rank):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2311_08872_gb300 import mlmc_dk

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    from paper_2311_08872_gb300 import distributed as D
    alloc = list(wl.alloc) if wl.alloc else None
    seed0 = wl.seed
    first0 = D.first_sample(rank)          # ranks shard the sample ids (no collective on the data path)

    ctx = mlmc_dk.Context.from_workload(wl, stream=stream.cuda_stream)
    tune_s = ctx.tune(repeats=1)          # autotuner: fastest kernel variant per level (outside timing)
    choice = ctx.variants()
    info = [ctx.level_info(l) for l in range(wl.L_max + 1)]

    # ---- a complete adaptive Algorithm 1 run, measured (at a looser eps than the
    #      workload's when the workload's eps would take longer than the bench allows)
    adaptive = None
    if not args.no_adaptive:
        eps_meas = args.adaptive_eps or wl.eps_rel
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = ctx.estimate(eps_meas, relative=True, seed=seed0 + 5)
        torch.cuda.synchronize()
        adaptive = {"eps_rel": eps_meas, "s": time.perf_counter() - t, "L": r.L,
                    "M": [r.M[l] for l in range(r.L + 1)], "estimate": r.estimate, "variance": r.variance,
                    "eps_abs": r.eps_abs, "converged": bool(r.converged), "cell_steps": r.cell_steps}
    if alloc is None:
        raise SystemExit("workload has no fixed allocation")
    alloc = alloc + [0] * (wl.L_max + 1 - len(alloc))
    sample_steps, cell_steps = batch_units(wl, alloc)
    # batch split: share of the 256^2 level's samples on the streamed kernels, on the
    # SMs its 8-SM clusters leave free (tuned on the batch itself, outside the timing)
    split_level = max((l for l in range(len(alloc)) if ctx.level_info(l).split_capable), default=None)
    if args.split_fraction is None:
        split_frac, split_s = ctx.tune_batch(alloc, 1)
    else:
        split_frac, split_s = args.split_fraction, 0.0
        if split_level is not None:
            ctx.set_batch_split(split_level, split_frac)

    nq = ctx.n_quant
    sums = torch.zeros(wl.L_max + 1, mlmc_dk.sums_len(nq), dtype=torch.float64, device=dev)
    host = torch.zeros_like(sums, device="cpu").pin_memory()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    step_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def step(seed):
        # all levels concurrently: one CUDA-graph launch of the multi-level batch
        step_ev[0].record(stream)
        ctx.run_batch_dev(alloc, first0, seed, sums.data_ptr(), stream.cuda_stream)
        host.copy_(sums, non_blocking=True)
        step_ev[1].record(stream)
        stream.synchronize()
        s = host.numpy()
        est, var = 0.0, 0.0
        for l, m in enumerate(alloc):
            if m <= 0:
                continue
            e = s[l, 2] / m
            est += e
            var += max(0.0, (s[l, 3] - s[l, 2] ** 2 / m) / (m - 1)) / m
        return est, var, s.copy()

    for w in range(args.warmup):
        step(seed0 + 17 + w)
    clocks = Clocks(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms, level_ms = [], [0.0] * len(alloc)
    launches = 0
    last = None
    for k in range(args.steps):
        flush.zero_()                      # evict L2 between steps (outside the step events)
        last = step(seed0 + 101 + k)
        step_ms.append(step_ev[0].elapsed_time(step_ev[1]))
        for l, t in enumerate(ctx.batch_level_ms()):   # CUDA events on each level's stream in the graph
            level_ms[l] += t
            if alloc[l] > 0:
                launches += 2
            d = ctx.level_info(l)
            if d.batch_streamed > 0:      # zero + per wave (init, fine steps, coarse steps, observe, finish) + reduce + merge
                waves = -(-d.batch_streamed // d.in_flight)
                launches += 1 + waves * (3 + d.M + d.M // 4) + 2
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * sample_steps * args.steps / (total_ms * 1e-3)

    split_samples = ctx.level_info(split_level).batch_streamed if split_level is not None else 0

    # ---- roofline of the dominant kernel (the level kernel of the costliest level)
    dom = max(range(len(alloc)), key=lambda l: level_ms[l])
    if level_ms[dom] <= 0:
        raise SystemExit("no per-level kernel times from the batch")
    lv, fine, coarse = level_costs(wl)
    reg_dom = alloc[dom] - ctx.level_info(dom).batch_streamed    # samples the register kernel ran
    ops = reg_dom * (fine[dom] * XU_OPS_FINE + coarse[dom] * XU_OPS_COARSE) * args.steps
    achieved = ops / (level_ms[dom] * 1e-3)
    peak = XU_PER_CLK_PER_SM * SMS * SM_MAX_MHZ * 1e6
    kname = (f"level_kernel n={info[dom].n} C={info[dom].lane_cols} R={info[dom].lane_rows} "
             f"cluster={info[dom].cluster} coupled={dom > 0}")
    traffic = None
    if kname == LEVEL_KERNEL_TRAFFIC["kernel"] and kernel_sources_hash() == LEVEL_KERNEL_TRAFFIC["sources_sha256_16"]:
        traffic = LEVEL_KERNEL_TRAFFIC["bytes_per_launch"]
    issue = None
    if traffic is not None:   # same sources as the capture that counted the instructions
        warp_inst = reg_dom * fine[dom] * LEVEL_KERNEL_INSTR_PER_CELL_STEP / 32.0 * args.steps / (level_ms[dom] * 1e-3)
        issue = {"instructions_per_fine_cell_step": LEVEL_KERNEL_INSTR_PER_CELL_STEP,
                 "achieved_warp_inst_per_s": warp_inst, "peak_all_sms": 4 * SMS * SM_MAX_MHZ * 1e6,
                 "frac_all_sms": warp_inst / (4 * SMS * SM_MAX_MHZ * 1e6),
                 "note": "instruction-issue roofline: the binding limit; the clusters of 8 hold 120 of 152 SMs"}
    roofline = {"bound": "alu", "pipe": "XU (MUFU)",
                "kernel": kname,
                "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gop/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_unit": "DRAM bytes per launch (ncu, one launch per step)",
                "ops_per_fine_cell_step": XU_OPS_FINE,
                "samples_per_launch": reg_dom,
                "issue": issue,
                "cell_steps_per_s": reg_dom * (fine[dom] + coarse[dom]) * args.steps / (level_ms[dom] * 1e-3),
                "level_ms_per_step": [x / args.steps for x in level_ms],
                "note": "levels run concurrently in one CUDA graph; each level's time is its own stream's span"}

    # ---- time to the workload's eps, MLMC against plain MC on the finest level.
    # From the timed batch: V_l = Var[P_l - P_{l-1}]; the eps-optimal cost in
    # cell-steps is 2 eps^-2 (sum_l sqrt(V_l C_l))^2 (Eq. opt_M_ell with C_l the
    # cell-steps of one coupled sample, as Algorithm 1 uses), timed at the
    # batch's measured cell-step rate; plain MC needs 2 Var[P_L] / eps^2
    # samples of level L, timed separately below.
    est, _, s = last
    Ls = max(l for l, m in enumerate(alloc) if m > 0)
    V, C = [], []
    for l, m in enumerate(alloc):
        if m > 0:
            V.append(max(0.0, (s[l, 3] - s[l, 2] ** 2 / m) / (m - 1)))
            C.append(fine[l] + coarse[l])
    eps_abs = wl.eps_rel * abs(est)
    cost_opt = 2.0 / eps_abs ** 2 * sum(math.sqrt(v * c) for v, c in zip(V, C)) ** 2
    rate = cell_steps * args.steps / (sum(step_ms) * 1e-3)
    t_mlmc = cost_opt / rate
    mL = alloc[Ls]
    var_pL = max(0.0, (s[Ls, 7] - s[Ls, 6] ** 2 / mL) / (mL - 1))
    n_mc = int(max(32, min(20000, 2.0e11 / fine[Ls])))
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    ctx.run_level(Ls, n_mc, seed0 + 7, mc=True)
    a1.record(stream)
    torch.cuda.synchronize()
    per = a0.elapsed_time(a1) * 1e-3 / n_mc
    m_mc = math.ceil(2.0 * var_pL / eps_abs ** 2)
    mc = {"level": Ls, "samples": m_mc, "s_per_sample": per, "s": m_mc * per, "extrapolated": True,
          "measured_samples": n_mc, "var_P_L": var_pL}
    to_eps = {"eps_rel": wl.eps_rel, "eps_abs": eps_abs, "estimate": est, "V": V, "cost_cell_steps": cost_opt,
              "batch_cell_steps_per_s": rate, "mlmc_s": t_mlmc, "mc_s": m_mc * per, "extrapolated": True,
              "how": "eps-optimal cost from the timed batch's V_l at its measured cell-step rate; "
                     "plain MC from 2 Var[P_L]/eps^2 samples at the measured MC time per sample"}

    # ---- learned level below 0 (trained on 2^18 level-0 paths): the same eps-optimal
    #      time with levels {S, P_0 - S, 1..L} in place of {0, 1..L}
    surrogate = None
    if not args.no_surrogate:
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx.surrogate_init(seed0 + 3)
        tr = ctx.surrogate_train(1 << 18, epochs=8, batch=1024, lr=1e-3, seed=seed0 + 4)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t
        n_s = 200000
        s_sur = ctx.run_surrogate(-1, n_s, seed0 + 5)[0]
        s_cor = ctx.run_surrogate(0, n_s, seed0 + 6)[0]
        var = lambda q: max(0.0, (q.dp2 - q.dp1 ** 2 / q.n) / (q.n - 1))
        t_l = [c / rate for c in C]        # seconds per sample of levels 0..L at the batch's rate
        terms = [math.sqrt(var(s_sur) * s_sur.kernel_s / n_s), math.sqrt(var(s_cor) * s_cor.kernel_s / n_s)]
        terms += [math.sqrt(v * tt) for v, tt in zip(V[1:], t_l[1:])]
        t_sur = 2.0 / eps_abs ** 2 * sum(terms) ** 2
        surrogate = {"train_s": train_s, "train_pairs": 1 << 18, "val_mse": tr["val_mse"],
                     "var_P0": V[0], "var_S": var(s_sur), "var_P0_minus_S": var(s_cor),
                     "s_per_sample_S": s_sur.kernel_s / n_s, "s_per_sample_P0_minus_S": s_cor.kernel_s / n_s,
                     "s_per_sample_P0": t_l[0], "mlmc_s_to_eps": t_sur,
                     "mlmc_s_to_eps_incl_training": t_sur + train_s, "extrapolated": True}

    streamed = None
    if not args.no_streamed:
        streamed = streamed_stencil(stream)
    theta = None
    if not args.no_theta:
        theta = theta_scheme(stream)
    fourier = None
    if not args.no_fourier:
        fourier = fourier_coupling(stream)

    e2e = None
    if not args.no_e2e:
        ctx.close()
        times, h2d, d2h = [], 0, 0
        for k in range(args.steps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            c2 = mlmc_dk.Context.from_workload(wl, stream=stream.cuda_stream)
            for l, (vs, vc) in enumerate(choice):   # the tuned variants, as a user would reuse them
                c2.set_variant(l, False, vs)
                if l > 0:
                    c2.set_variant(l, True, vc)
            if split_level is not None:
                c2.set_batch_split(split_level, split_frac)
            res = c2.run_batch(alloc, seed0 + 101 + k)      # host sums of every level
            est = sum(res[l][0].dp1 / res[l][0].n for l, m in enumerate(alloc) if m > 0)
            d2h_k = 8 * mlmc_dk.sums_len(nq) * len(alloc) + 4
            h2d_k = c2.level_info(0).h2d_bytes
            c2.close()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t)
            h2d, d2h = h2d_k, d2h_k
        tot = sum(times)
        if world > 1:
            t = torch.tensor([tot], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            tot = float(t.item())
        e2e = {"value": world * sample_steps * args.steps / tot, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * tot / args.steps,
               "what": "mlmc_dk_init (FFT mean fields + pinned uploads) + mlmc_dk_run_batch (host sums) + free"}
    else:
        ctx.close()

    if rank != 0:
        return None
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_rate(wl, alloc, args.cpu_budget)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32 fixed-point state, f32 noise, f64 sums",
        "data": "synthetic",
        "config": {"workload": wl.name, "levels": [i.n for i in info], "fine_steps": [i.M for i in info],
                   "T": wl.T, "N": wl.N, "mu": wl.mu, "eps_rel": wl.eps_rel, "alloc": alloc,
                   "sample_steps_per_step": sample_steps, "cell_steps_per_step": cell_steps,
                   "l2": "512 MiB buffer zeroed between timed steps, outside the step events",
                   "parallelism": f"{world} rank(s), disjoint sample ids per rank",
                   "kernel_variants": [{"n": i.n, "C": i.lane_cols, "R": i.lane_rows, "cluster": i.cluster}
                                       for i in info],
                   "tune_s": tune_s,
                   "batch_split": {"level": split_level, "fraction": split_frac,
                                   "streamed_samples": split_samples, "tune_s": split_s}},
        "cell_steps_per_s": world * cell_steps * args.steps / (total_ms * 1e-3),
        "gpu_launches": launches,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
    }
    line["mlmc_s_to_eps"] = t_mlmc
    line["mc_s_to_eps"] = mc["s"]
    line["mlmc_speedup_vs_mc"] = mc["s"] / t_mlmc
    line["to_eps"] = to_eps
    line["mc"] = mc
    line["mlmc_adaptive_measured"] = adaptive
    fin = info[Ls]
    cf = closed_form_EP_cos1(fin.n, fin.tau, fin.M) if wl.rho0_kind == "sinsin" and wl.length == 1.0 else None
    line["closed_form_EP_finest"] = {"value": cf, "estimate": to_eps["estimate"],
                                     "note": "martingale-lemma E[P_L] if rho stayed positive; at the finest "
                                             "level N h^2 = %.2g particles per cell, so it is a lower bound and "
                                             "the gap is the positive-part effect" % (wl.N * (wl.length / fin.n) ** 2)}
    line["streamed_stencil"] = streamed
    line["theta_scheme"] = theta
    line["fourier_coupling"] = fourier
    if surrogate:
        line["surrogate"] = surrogate
        line["mlmc_surrogate_s_to_eps"] = surrogate["mlmc_s_to_eps_incl_training"]
    return line


def run_reference(args, wl, rank, world):
    if rank != 0:
        return None
    alloc = list(wl.alloc) if wl.alloc else None
    if alloc is None:
        return {"impl": "reference", "unavailable": "workload has no fixed allocation"}
    alloc = alloc + [0] * (wl.L_max + 1 - len(alloc))
    sample_steps, cell_steps = batch_units(wl, alloc)
    budget = max(2.0, args.cpu_budget / 3)
    for _ in range(args.warmup):
        oracle_rate(wl, alloc, budget / 2)
    vals, res = [], None
    for _ in range(args.steps):
        res = oracle_rate(wl, alloc, budget)
        vals.append(res["batch_cpu_s"])
    cpu_s = statistics.mean(vals)
    value = sample_steps / cpu_s
    cb = dict(res)
    cb["value"] = value
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * cpu_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "alloc": alloc, "sample_steps_per_step": sample_steps,
                       "cell_steps_per_step": cell_steps,
                       "what": "FP64 oracle (plain C) per coupled sample on the host cores; each step times a "
                               "bounded sample of the batch and scales it to the full batch by level"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    from paper_2311_08872_gb300 import workloads
    wl = workloads.get(args.workload)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, wl, rank, world)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        line = run_ours(args, wl, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
