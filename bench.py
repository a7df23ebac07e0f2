#!/usr/bin/env python3
"""Benchmark of the GB300 MLMC hot path for the 2-D Dean--Kawasaki equation.

Workload (default ``large32_1024``, the largest single-GPU configuration):
unit torus, levels 32^2..1024^2 (h_l = 1/32..1/1024, six levels), tau_l =
0.1 h_l^2 (tau_0 = 9.766e-5, 512..524288 fine steps), T = 0.05, N = 1e6,
rho0 = 1 + 0.5 sin sin + 0.3 cos(4 pi x2), observables (rho_T, cos 2 pi k.x)_h
for k in {(1,0), (0,1), (1,1), (2,0)} with all ten pairwise products, NN-coupled
levels, the learned level below level 0, RMSE target eps = 5e-4 relative.

One *step* is one pass of the whole hot path over the workload's MLMC batch:
the eps-optimal allocation (Eq. opt_M_ell, from pilot variances, divided by
2^20) of coupled samples on levels 1..5 (Philox normals, fused fine/coarse
stepping, observables, P, FP64 moment sums; the register levels in one CUDA
graph, the band-kernel levels beside it), plus the learned level's two parts
(the level below 0 drawn from its exact feature law and the correction level
P_0 - S on level-0 paths through the BF16 network), then the estimator and its
variance from the sums (Eq. MLMCEstimator).  ``value`` is coupled sample-steps
per second (sum over levels of samples x fine steps, the correction level
counted with level 0's steps), inputs resident on the device; ``e2e`` is the
same through the public C-ABI with host buffers (init uploads the level tables
and the trained network from pinned memory, host sums are read back).

Under torchrun every rank runs the same batch on its own sample ids
(independent samples, no collective on the data path): weak scaling.
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
KERNEL_SOURCES = ("dk_kernels.cu", "dk_device.cuh")   # the register kernel and its device functions
BAND_SOURCES = ("dk_band.cu", "dk_device.cuh")


# Theta-scheme kernel (implicit diffusion weight b0 > 0): thread instructions
# per fine cell-step (coupled, coarse work included) of the 64^2 coupled
# launch at b0 = 1/2, tau/h^2 = 0.85 (14 Chebyshev steps per solve), from its
# ncu --set full capture (smsp__inst_executed x 32 / fine cell-steps); valid
# under the recorded hash of its sources.  Bound by instruction issue.
THETA_KERNEL_INSTR = {"kernel": "theta_kernel n=64 coupled=True b0=0.5 chebyshev_steps=14",
                      "instructions_per_fine_cell_step": 580.6, "sources_sha256_16": "e8dc915d7d236c06"}
THETA_SOURCES = ("dk_theta.cu", "dk_device.cuh")
# Fourier-coupled kernel: thread instructions per cell-step (fine and coarse
# cell-steps) of the 54^2 coupled launch, from its ncu --set full capture;
# valid under the recorded hash of its sources.
FOURIER_KERNEL_INSTR = {"kernel": "fourier_kernel n=54 coupled=True",
                        "instructions_per_cell_step": 94.6, "sources_sha256_16": "f3dd0738e5d2295f"}
FOURIER_SOURCES = ("dk_fourier.cu", "dk_device.cuh")
# The 162^2 Fourier level on 6-CTA clusters: thread instructions per cell-step
# (fine and coarse cell-steps) of the coupled launch of 144 samples, from its
# ncu capture; valid under the recorded hash of its sources.
FOURIER_CLUSTER_KERNEL_INSTR = {"kernel": "fourier_cluster_kernel n=162 coupled=True",
                                "instructions_per_cell_step": 106.7, "sources_sha256_16": "9d8da938f719df45"}
FOURIER_CLUSTER_SOURCES = ("dk_fourier_cluster.cu", "dk_device.cuh")


# ncu figures of the dominant kernels per grid size, valid while their sources
# hash to the recorded value: DRAM bytes (read + write) per fine cell-step of a
# warm-cache launch (--cache-control none, so the L2-resident working set stays
# resident as in the bench) and thread instructions per fine cell-step
# (smsp__inst_executed x 32 / fine cell-steps); keyed by kernel function.
KERNEL_PROFILE = {
    "stream_fine_kernel": {
        "sources": ("dk_stream.cu", "dk_device.cuh"), "sources_sha256_16": "4a364a9befb1c264",
        "per_n": {1024: {"dram_bytes_per_fine_cell_step": 0.92, "instructions_per_fine_cell_step": 82.8},
                  512: {"dram_bytes_per_fine_cell_step": 0.016, "instructions_per_fine_cell_step": 82.8}},
        "capture": "ncu --cache-control none, 3 consecutive launches of the 1024^2 (5 samples) and 512^2 "
                   "(8 samples) fine step (profiles/stream_fine_kernel_1024_pdl_full.md, _512_pdl_full.md)",
    },
}


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
    """(HBM GB/s, source) from the measured peaks file, else the fallback."""
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
    """The 512^2 level of the low-density workload (coupled with 256^2, 52480
    fine steps): one launch group of the samples in flight on the level's tuned
    large-grid kernel (the band kernel unless the tuner prefers the streamed
    state), CUDA events on the launching stream, against the HBM rate a state
    streamed through memory would need (8.5 algorithmic bytes per coupled fine
    cell-step)."""
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
    kernel = f"band_kernel bands={info.bands}" if info.band else f"streamed tile_rows={info.tile_rows}"
    return {"workload": wl.name, "level": level, "n": info.n, "fine_steps": info.M, "samples": S, "kernel": kernel,
            "s": sec, "cell_steps_per_s": S * info.cost / sec,
            "fine_cell_steps_per_s": fine / sec, "algorithmic_bytes_per_fine_cell_step": STREAM_BYTES_PER_FINE_CELL_STEP,
            "achieved_GBps": gbs, "hbm_peak_GBps": peak, "peak_source": src, "frac_of_hbm": gbs / peak,
            "bound": "alu (instruction issue): the state stays on chip; DRAM sees the tables only"}


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
    coupled with 18^2, ratio 3): 32 waves of one sample per SM, CUDA events;
    and the 162^2 level of fourier6_162 (coupled with 54^2) on its cluster
    kernel, 144 samples."""
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
    # the 162^2 level (coupled with 54^2) on 6-CTA clusters, 144 samples in one launch
    wl = workloads.get("fourier6_162")
    level, count = wl.L_max, 144
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
    cl = {"workload": wl.name, "level": level, "n": info.n, "coarse_n": info.n // 3, "fine_steps": info.M,
          "cluster": info.cluster, "samples": count, "s": sec, "cell_steps_per_s": count * info.cost / sec,
          "fine_cell_steps_per_s": count * info.cost_mc / sec, "coupled_sample_steps_per_s": count * info.M / sec,
          "bound": "alu (instruction issue; shared-memory queue and scoreboard stalls lead)"}
    if kernel_sources_hash(FOURIER_CLUSTER_SOURCES) == FOURIER_CLUSTER_KERNEL_INSTR["sources_sha256_16"]:
        ipc = FOURIER_CLUSTER_KERNEL_INSTR["instructions_per_cell_step"]
        warp_inst = count * info.cost * ipc / 32.0 / sec
        peak = 4.0 * SMS * SM_MAX_MHZ * 1e6
        cl["issue"] = {"instructions_per_cell_step": ipc, "achieved_warp_inst_per_s": warp_inst,
                       "peak_warp_inst_per_s": peak, "frac": warp_inst / peak}
    out["cluster_162"] = cl
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="large32_1024")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-streamed", action="store_true", help="skip the streamed-state stencil timing")
    ap.add_argument("--no-theta", action="store_true", help="skip the theta-scheme kernel timing")
    ap.add_argument("--no-fourier", action="store_true", help="skip the Fourier-coupled kernel timing")
    ap.add_argument("--split-fraction", type=float, default=None,
                    help="fixed batch split of the finest cluster level (default: autotuned)")
    ap.add_argument("--profile-level", default=None, metavar="WORKLOAD:LEVEL:SAMPLES[:T[:VARIANT]]",
                    help="run one level batch twice (a small case for a profiler), print its timing and exit")
    ap.add_argument("--profile-gemm", type=int, default=0, metavar="ROWS",
                    help="run the learned level's network forward on ROWS rows twice (tensor-core GEMMs) and exit")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary measurements (16^2..256^2 batch, 512^2 stencil, theta, Fourier)")
    ap.add_argument("--no-mlmc16", action="store_true", help="skip the 16^2..256^2 batch and Algorithm 1 run")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned level below 0")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default kernel variants and no batch split (profiling runs: timings taken "
                         "under a profiler would mislead the tuner)")
    ap.add_argument("--t-scale", type=float, default=1.0,
                    help="divide the workload's T by this (profiling runs: the same levels and launch mix "
                         "with fewer steps; the line then describes that shorter workload)")
    ap.add_argument("--adaptive-eps", type=float, default=1e-2,
                    help="relative eps of the fully measured Algorithm 1 run (0: the workload's)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def nominal_levels(wl):
    """(n_l, M_l) of the workload's hierarchy: M_0 = ceil(T / (mu h_0^2)), M_l =
    M_0 4^l (labels of the config; the work units come from the library's or
    the oracle's own level table)."""
    h0 = wl.length / wl.n0
    x = wl.T / (wl.mu * h0 * h0)
    M0 = wl.M0 or int(math.ceil(x - 1e-9 * x))
    return [(wl.n0 * 2 ** l, M0 * 4 ** l) for l in range(wl.L_max + 1)]


def workload_config(wl, alloc, learned):
    lv = nominal_levels(wl)
    cfg = {"workload": wl.name, "levels": [n for n, _ in lv], "fine_steps": [m for _, m in lv], "T": wl.T, "N": wl.N,
           "mu": wl.mu, "n_obs": len(wl.observables), "products": bool(wl.products), "eps_rel": wl.eps_rel,
           "alloc": list(alloc), "alloc_scale": wl.alloc_scale}
    if learned is not None:
        cfg["alloc_learned"] = {"below_0": learned[0], "correction": learned[1]}
    return cfg


def step_units(fine, coarse, M, alloc, learned):
    """Coupled sample-steps and cell-steps of one step: levels l >= 1 from
    alloc, level 0 from alloc[0] or, with the learned level, the correction
    level's count (its level-0 paths; the level below 0 takes no steps)."""
    n0 = alloc[0] if learned is None else learned[1]
    sample_steps = n0 * M[0] + sum(alloc[l] * M[l] for l in range(1, len(alloc)))
    cell_steps = n0 * fine[0] + sum(alloc[l] * (fine[l] + coarse[l]) for l in range(1, len(alloc)))
    return sample_steps, cell_steps


def oracle_level_costs(wl):
    import oracle
    lv = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu, wl.M0)
    fine = [l.n * l.n * l.M for l in lv]
    coarse = [0.0] + [lv[l - 1].n ** 2 * lv[l - 1].M for l in range(1, len(lv))]
    return [l.M for l in lv], fine, coarse


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
    (wl, level, sample, seed) = args
    import oracle
    lv = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu, wl.M0)
    ol = oracle.level_inputs(wl.length, lv, wl.N, wl.rho0_all(), wl.phi_all(), level, level > 0)
    t = time.perf_counter()
    r = ol.sample(seed, sample, level > 0)
    dt = time.perf_counter() - t
    return level, sample, dt, list(r["Y_f"]), (list(r["Y_c"]) if level > 0 else None)


def oracle_leg(wl, alloc, learned, budget_s, seed, first, cores=None):
    """The FP64 oracle, as it stands, on the host cores (one process per core,
    each single-threaded): coupled samples with the benchmark step's own seed
    and sample ids on every level whose samples fit the budget (a bounded
    sample of the workload), timed per level and extrapolated by cell-steps to
    the others.  Returns the timing figures and the oracle's per-sample
    observables (for the per-sample error of the GPU path on the same ids)."""
    import multiprocessing as mp
    nproc = os.cpu_count() or 1
    cores = cores or min(nproc, 16)
    M, fine, coarse = oracle_level_costs(wl)
    per_cell = 1.0 / 2.5e7     # first guess (one core), refined by the measurement
    tasks = []
    for l in range(len(alloc)):
        est = (fine[l] + coarse[l]) * per_cell
        if est > budget_s * cores / 6:
            continue
        k = max(1, min(64, cores, int(budget_s * cores / (4 * max(est, 1e-6) * len(alloc)))))
        if l > 0 and k < 2 and est > budget_s / 2:
            k = 1
        tasks += [(wl, l, first + i, seed) for i in range(k)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_task, tasks, chunksize=1)
    wall = time.perf_counter() - t0
    per_level, outs = {}, {}
    for l, i, dt, yf, yc in res:
        per_level.setdefault(l, []).append(dt)
        outs.setdefault(l, {})[i] = (yf, yc)
    t = {l: statistics.mean(v) for l, v in per_level.items()}
    top = max(t)
    cell_rate = (fine[top] + coarse[top]) / t[top]
    secs = [0.0] * len(alloc)
    for l, m in enumerate(alloc):
        if l == 0 and learned is not None:
            m = learned[1]     # the correction level's level-0 paths (network cost not counted)
        secs[l] = m * (t[l] if l in t else (fine[l] + coarse[l]) / cell_rate)
    sample_steps, cell_steps = step_units(fine, coarse, M, alloc, learned)
    cpu_time = sum(secs) / cores
    sample = (f"{len(tasks)} coupled samples (the step's seed and ids) of levels {sorted(t)} in {wall:.1f} s wall "
              f"on {cores} processes; levels {[l for l in range(len(alloc)) if l not in t]} extrapolated by "
              f"cell-steps from level {top}")
    return {"value": sample_steps / cpu_time, "unit": UNIT, "cores": cores, "nproc": nproc, "kind": "oracle",
            "sample": sample, "cell_steps_per_s": cell_steps / cpu_time,
            "cell_steps_per_s_per_core": cell_steps / cpu_time / cores,
            "batch_cpu_s": cpu_time, "wall_s": wall}, outs


def level_launches(d, count, coupled):
    """Kernel launches of one level's share of a batch, from its kernel's description."""
    if d.band:                                   # zero + per wave (kernel + finish) + reduce
        return 2 + 2 * (-(-count // d.in_flight))
    if d.streamed:                               # zero + per wave (init, steps, observe, finish) + reduce
        steps = 1 if d.persistent else d.M + (d.M // 4 if coupled else 0)
        return 2 + (-(-count // d.in_flight)) * (3 + steps)
    n = 2                                        # level kernel + reduce
    if d.batch_streamed > 0:                     # the split share: one launch per step, then the merge
        n += 2 + (-(-d.batch_streamed // d.in_flight)) * (3 + d.M + d.M // 4) + 1
    return n


def oracle_samples(wl, counts, seed, cores=None):
    """The FP64 oracle's observables for ids 0..counts[l]-1 of each level
    (coupled), one process per core: {level: {id: (Y_f, Y_c)}}."""
    import multiprocessing as mp
    cores = cores or min(os.cpu_count() or 1, 16)
    tasks = [(wl, l, i, seed) for l, k in enumerate(counts) for i in range(k)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_task, tasks, chunksize=1)
    outs = {}
    for l, i, _, yf, yc in res:
        outs.setdefault(l, {})[i] = (yf, yc)
    return outs


def network_error(ctx, theta, outputs, rows, seed):
    """The learned level's network (BF16 operands, FP32 accumulation, tensor
    cores) against the same network in FP64 on the level's own feature rows:
    max and RMS of |y_gpu - y_fp64| over RMS(y_fp64)."""
    import numpy as np
    from oracle import surrogate as sg
    X = ctx.surrogate_features(0, rows, seed, direct=True)
    y = ctx.surrogate_forward(X).astype(np.float64).reshape(rows, -1)
    yo, _ = sg.mlp_forward(theta.astype(np.float64), X.astype(np.float64), outputs)
    yo = yo.reshape(rows, -1)
    scale = np.sqrt(np.mean(yo ** 2, axis=0))
    d = np.abs(y - yo) / scale[None, :]
    return {"rows": rows, "max_err_over_rms": float(d.max()), "rms_err_over_rms": float(np.sqrt(np.mean(d ** 2))),
            "what": "network outputs on directly drawn level -1 feature rows against the FP64 network with the "
                    "same parameters; the BF16 rounding of the operands sets this error, and the correction "
                    "level E[P_0 - S] removes its effect on the estimate (the estimator stays unbiased)"}


def oracle_error(ctx, wl, outs, seed, stream):
    """Per-sample error of the GPU path against the oracle on the same ids:
    max |Y_gpu - Y_oracle| / max(|Y_oracle|, RMS of the level's Y_oracle - Ybar)
    over the observables of the fine and coarse paths, and the level means of
    P_l - P_{l-1} (every quantity) from both on those ids."""
    import numpy as np
    import torch
    from paper_2311_08872_gb300 import mlmc_dk
    K = ctx.n_obs
    rows = []
    worst = 0.0
    for l in sorted(outs):
        ids = sorted(outs[l])
        first, k = ids[0], len(ids)
        assert ids == list(range(first, first + k))
        info = ctx.level_info(l)
        sums = torch.zeros(mlmc_dk.sums_len(ctx.n_quant), dtype=torch.float64, device="cuda")
        samp = torch.zeros(k, mlmc_dk.sample_stride(K), dtype=torch.float64, device="cuda")
        ctx.run_level_dev(l, 0, first, k, seed, sums.data_ptr(), samp.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        g = samp.cpu().numpy()
        yf_o = np.array([outs[l][i][0] for i in ids])
        yb_f = np.array(info.ybar_f[:K])
        pairs = [(g[:, :K] + yb_f[None, :], yf_o, yb_f)]
        if l > 0:
            yc_o = np.array([outs[l][i][1] for i in ids])
            yb_c = np.array(info.ybar_c[:K])
            pairs.append((g[:, K:2 * K] + yb_c[None, :], yc_o, yb_c))
        lw = 0.0
        for yg, yo, yb in pairs:
            scale = np.sqrt(np.mean((yo - yb[None, :]) ** 2, axis=0))
            lw = max(lw, float(np.max(np.abs(yg - yo) / np.maximum(np.abs(yo), scale[None, :]))))
        worst = max(worst, lw)

        def dP(Df, Dc):
            cols = []
            for j in range(K):
                for q in range(j, K if wl.products else j + 1):
                    pf = wl.N * Df[:, j] * Df[:, q]
                    pc = wl.N * Dc[:, j] * Dc[:, q] if Dc is not None else 0.0
                    cols.append(pf - pc)
            return np.stack(cols, axis=1)
        dg = dP(g[:, :K], g[:, K:2 * K] if l > 0 else None)
        do = dP(yf_o - yb_f[None, :], (yc_o - yb_c[None, :]) if l > 0 else None)
        rows.append({"level": l, "n": info.n, "ids": [first, first + k - 1], "max_err_over_bar_scale": lw,
                     "mean_dP_gpu": dg.mean(axis=0).tolist(), "mean_dP_oracle": do.mean(axis=0).tolist(),
                     "max_abs_diff_mean_dP": float(np.max(np.abs(dg.mean(axis=0) - do.mean(axis=0))))})
    return {"levels": rows, "worst_err_over_bar_scale": worst, "bar": 1e-5,
            "within_bar": worst <= 1e-5,
            "what": "per-sample |Y_gpu - Y_oracle| / max(|Y_oracle|, RMS(Y_oracle - Ybar)) on the step's seed and ids "
                    "of the levels the oracle finished (FP32 noise and 32-bit fixed-point state against FP64); "
                    "the per-sample bar is 1e-5 of that scale; the level means of dP from both on the same ids",
            "levels_without_oracle": "finer levels: the oracle needs hours per sample there; their kernels are "
                                     "checked against the oracle over short horizons and against each other "
                                     "(tests/test_gpu_band.py, tests/test_gpu_stream.py)"}


# --------------------------------------------------------------- our arm
def run_ours(args, wl, rank, world, local_rank):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2311_08872_gb300 import distributed as D
    from paper_2311_08872_gb300 import mlmc_dk

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    if wl.alloc is None:
        raise SystemExit("workload has no fixed allocation")
    L = wl.L_max
    alloc = list(wl.alloc) + [0] * (L + 1 - len(wl.alloc))
    learned = tuple(wl.alloc_learned) if (wl.alloc_learned and not args.no_surrogate) else None
    seed0 = wl.seed
    first0 = D.first_sample(rank)          # ranks shard the sample ids (no collective on the data path)

    ctx = mlmc_dk.Context.from_workload(wl, stream=stream.cuda_stream)
    tune_s = 0.0 if args.no_tune else ctx.tune(repeats=1)   # autotuner: fastest kernel per level (outside timing)
    choice = ctx.variants()
    info = [ctx.level_info(l) for l in range(L + 1)]
    M = [i.M for i in info]
    fine = [i.cost_mc for i in info]
    coarse = [i.cost - i.cost_mc for i in info]
    sample_steps, cell_steps = step_units(fine, coarse, M, alloc, learned)
    nq = ctx.n_quant

    # the learned level below 0 is trained once, outside the timed region: the
    # network is an input of every step (like the level tables)
    sur = None
    theta = None
    if learned is not None:
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx.surrogate_init(seed0 + 3)
        tr = ctx.surrogate_train(1 << 18, epochs=8, batch=1024, lr=1e-3, seed=seed0 + 4)
        torch.cuda.synchronize()
        sur = {"train_s": time.perf_counter() - t, "train_pairs": 1 << 18, "val_mse": tr["val_mse"]}
        theta = ctx.surrogate_params()

    batch_counts = list(alloc)
    if learned is not None:
        batch_counts[0] = 0
    # batch split: a share of an 8-SM-cluster level's samples on the streamed
    # kernels (only where such a level runs the register kernel)
    split_level = max((l for l in range(L + 1) if info[l].split_capable and not info[l].band), default=None)
    split_frac, split_s = 0.0, 0.0
    if split_level is not None:
        if args.split_fraction is None:
            split_frac, split_s = (0.0, 0.0) if args.no_tune else ctx.tune_batch(batch_counts, 1)
        else:
            split_frac = args.split_fraction
            ctx.set_batch_split(split_level, split_frac)

    S = mlmc_dk.sums_len(nq)
    sums = torch.zeros(L + 1, S, dtype=torch.float64, device=dev)
    host = torch.zeros_like(sums, device="cpu").pin_memory()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    step_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def sur_array(parts):
        return np.array([[p.n, p.dp1, p.dp2, p.pf1, p.pf2, p.kernel_s, p.launches] for p in parts])

    def step(seed):
        step_ev[0].record(stream)
        ctx.run_batch_dev(batch_counts, first0, seed, sums.data_ptr(), stream.cuda_stream)
        parts = None
        if learned is not None:
            # the level below 0 and the correction level P_0 - S (host sums; same stream)
            parts = (sur_array(ctx.run_surrogate(-1, learned[0], seed)),
                     sur_array(ctx.run_surrogate(0, learned[1], seed)))
        host.copy_(sums, non_blocking=True)
        step_ev[1].record(stream)
        stream.synchronize()
        return host.numpy().copy(), parts

    def estimate(s, parts):
        """Eq. (MLMCEstimator) for every quantity, and its variance."""
        est, var = np.zeros(nq), np.zeros(nq)
        for l in range(L + 1):
            m = batch_counts[l]
            if m <= 1:
                continue
            d1, d2 = s[l, 2 + 12 * np.arange(nq)], s[l, 3 + 12 * np.arange(nq)]
            est += d1 / m
            var += np.maximum(0.0, (d2 - d1 * d1 / m) / (m - 1)) / m
        if parts is not None:
            for p in parts:
                n = p[:, 0]
                est += p[:, 1] / n
                var += np.maximum(0.0, (p[:, 2] - p[:, 1] ** 2 / n) / (n - 1)) / n
        return est, var

    for w in range(args.warmup):
        step(seed0 + 17 + w)
    clocks = Clocks(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms, level_ms = [], [0.0] * (L + 1)
    acc = np.zeros((L + 1, S))
    acc_parts = None
    launches = 0
    last = None
    for k in range(args.steps):
        flush.zero_()                      # evict L2 between steps (outside the step events)
        s, parts = step(seed0 + 101 + k)
        step_ms.append(step_ev[0].elapsed_time(step_ev[1]))
        acc += s
        if parts is not None:
            acc_parts = [p.copy() for p in parts] if acc_parts is None else [a + p for a, p in zip(acc_parts, parts)]
            launches += int(parts[0][0, 6] + parts[1][0, 6])
        last = (s, parts)
        for l, t in enumerate(ctx.batch_level_ms()):   # CUDA events on each level's stream
            level_ms[l] += t
            if batch_counts[l] > 0:
                launches += level_launches(ctx.level_info(l), batch_counts[l], l > 0)
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
    est, var = estimate(*last)

    # ---- roofline of the dominant kernel (the costliest level's kernel); the
    # streamed levels run concurrently on their own streams from one fork, so
    # their kernel is measured over all of them and their common span
    dom = max(range(L + 1), key=lambda l: level_ms[l])
    if level_ms[dom] <= 0:
        raise SystemExit("no per-level kernel times from the batch")
    dinfo = ctx.level_info(dom)
    group = [dom]
    if dinfo.streamed and not dinfo.band:
        group = [l for l in range(L + 1) if batch_counts[l] > 0 and ctx.level_info(l).streamed
                 and not ctx.level_info(l).band]
    ginfo = {l: ctx.level_info(l) for l in group}
    reg = {l: batch_counts[l] - ginfo[l].batch_streamed for l in group}
    sec_dom = max(level_ms[l] for l in group) * 1e-3
    fine_cs = sum(reg[l] * fine[l] for l in group) * args.steps
    all_cs = sum(reg[l] * (fine[l] + coarse[l]) for l in group) * args.steps
    xu_ops = sum(reg[l] * (fine[l] * XU_OPS_FINE + coarse[l] * XU_OPS_COARSE) for l in group) * args.steps
    xu_peak = XU_PER_CLK_PER_SM * SMS * SM_MAX_MHZ * 1e6
    hbm_peak, hbm_src = measured_peaks()
    if dinfo.band:
        kname = f"band_kernel n={dinfo.n} bands={dinfo.bands} in_flight={dinfo.in_flight} coupled={dom > 0}"
        family = "band_kernel"
    elif dinfo.streamed:
        how = "persistent" if dinfo.persistent else ("pdl" if dinfo.pdl else "per-step")
        family = "stream_persist_kernel" if dinfo.persistent else "stream_fine_kernel"
        kname = (f"{family} ({how}) n=" + ",".join(str(ginfo[l].n) for l in group) +
                 " in_flight=" + ",".join(str(ginfo[l].in_flight) for l in group) + " coupled=True")
    else:
        family = "level_kernel"
        kname = (f"level_kernel n={dinfo.n} C={dinfo.lane_cols} R={dinfo.lane_rows} "
                 f"cluster={dinfo.cluster} coupled={dom > 0}")
    traffic, issue = None, None
    rec = KERNEL_PROFILE.get(family)
    if rec and kernel_sources_hash(rec["sources"]) == rec["sources_sha256_16"] and \
            all(ginfo[l].n in rec["per_n"] for l in group):
        per_l = {l: reg[l] * fine[l] * args.steps for l in group}     # fine cell-steps of each level
        traffic = sum(per_l[l] * rec["per_n"][ginfo[l].n]["dram_bytes_per_fine_cell_step"] for l in group)
        inst = sum(per_l[l] * rec["per_n"][ginfo[l].n]["instructions_per_fine_cell_step"] for l in group)
        warp_inst = inst / 32.0 / sec_dom
        issue = {"instructions_per_fine_cell_step": inst / fine_cs, "achieved_warp_inst_per_s": warp_inst,
                 "peak_warp_inst_per_s": 4 * SMS * SM_MAX_MHZ * 1e6,
                 "frac": warp_inst / (4 * SMS * SM_MAX_MHZ * 1e6)}
    hbm_equiv = fine_cs * STREAM_BYTES_PER_FINE_CELL_STEP / sec_dom / 1e9
    roofline = {"bound": "alu", "pipe": "XU (MUFU)", "kernel": kname, "levels": group,
                "achieved": xu_ops / sec_dom / 1e9, "peak": xu_peak / 1e9, "unit": "Gop/s",
                "frac": xu_ops / sec_dom / xu_peak,
                "traffic": traffic,
                "traffic_unit": "DRAM bytes over the timed steps: ncu dram__bytes_read.sum + dram__bytes_write.sum "
                                "per fine cell-step of a warm-cache launch (small case, same kernel) x fine cell-steps",
                "ops_per_fine_cell_step": XU_OPS_FINE, "samples_per_step": sum(reg.values()),
                "cell_steps_per_s": all_cs / sec_dom, "fine_cell_steps_per_s": fine_cs / sec_dom,
                "issue": issue,
                "hbm_equivalent": {"algorithmic_bytes_per_fine_cell_step": STREAM_BYTES_PER_FINE_CELL_STEP,
                                   "achieved_GBps": hbm_equiv, "peak_GBps": hbm_peak, "peak_source": hbm_src,
                                   "frac": hbm_equiv / hbm_peak,
                                   "algorithmic_bytes_over_timed_steps": fine_cs * STREAM_BYTES_PER_FINE_CELL_STEP,
                                   "note": "the rate a state streamed through HBM would need; the streamed levels' "
                                           "working set stays in L2, so DRAM traffic (`traffic`) is far below it"},
                "level_ms_per_step": [x / args.steps for x in level_ms],
                "note": "XU ops are the algorithmic MUFU operations (Box--Muller log, sqrt, sin, cos; sqrt of rho+); "
                        "peak 16 per clock per SM x 152 SMs x 2.07 GHz; time = the span of the levels' kernels "
                        "(CUDA events on their streams)"}

    # ---- time to the workload's eps: plain MLMC, MLMC with the learned level, plain MC
    rate = cell_steps * args.steps / (sum(step_ms) * 1e-3)        # the batch's cell-steps per second
    t_l = [(fine[l] + coarse[l]) / rate for l in range(L + 1)]
    V = np.zeros((L + 1, nq))
    for l in range(1, L + 1):
        m = batch_counts[l] * args.steps
        if m > 1:
            d1, d2 = acc[l, 2 + 12 * np.arange(nq)], acc[l, 3 + 12 * np.arange(nq)]
            V[l] = np.maximum(0.0, (d2 - d1 * d1 / m) / (m - 1))
    n0p = 20000                                                    # level 0 of plain MLMC, measured apart
    s0 = ctx.run_level(0, n0p, seed0 + 9)
    V[0] = [max(0.0, (q.dp2 - q.dp1 ** 2 / q.n) / (q.n - 1)) for q in s0]
    est0 = np.array([q.dp1 / q.n for q in s0])
    plain_est = est.copy()
    if learned is not None:
        plain_est = est - sum(p[:, 1] / p[:, 0] for p in last[1]) + est0
    eps_abs = wl.eps_rel * float(np.max(np.abs(plain_est)))

    def opt_cost(Vs, ts):
        Mopt = np.zeros(len(ts))
        for q in range(nq):
            tot = sum(math.sqrt(v * t) for v, t in zip(Vs[:, q], ts))
            for i, (v, t) in enumerate(zip(Vs[:, q], ts)):
                if v > 0:
                    Mopt[i] = max(Mopt[i], math.ceil(2.0 / eps_abs ** 2 * math.sqrt(v / t) * tot))
        return Mopt, float(sum(m * t for m, t in zip(Mopt, ts)))

    M_plain, t_mlmc = opt_cost(V, t_l)
    # plain MC on the finest level: at least one full wave of samples in flight
    d_L = ctx.level_info(L)
    n_mc = max(2, int(2e11 / fine[L]), d_L.in_flight if (d_L.streamed or d_L.band) else 0)
    if fine[L] > 1e11:
        n_mc = max(1, d_L.in_flight)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    ctx.run_level(L, n_mc, seed0 + 7, mc=True)
    a1.record(stream)
    torch.cuda.synchronize()
    t_mc = a0.elapsed_time(a1) * 1e-3 / n_mc
    mL = batch_counts[L] * args.steps
    pf1, pf2 = acc[L, 6 + 12 * np.arange(nq)], acc[L, 7 + 12 * np.arange(nq)]
    var_pL = np.maximum(0.0, (pf2 - pf1 ** 2 / mL) / (mL - 1))
    m_mc = int(max(math.ceil(2.0 * v / eps_abs ** 2) for v in var_pL))
    to_eps = {"eps_rel": wl.eps_rel, "eps_abs": eps_abs, "estimate": plain_est.tolist(), "V": V[:, 0].tolist(),
              "M_opt": M_plain.tolist(), "batch_cell_steps_per_s": rate, "mlmc_s": t_mlmc,
              "mc_samples": m_mc, "mc_s_per_sample": t_mc, "mc_s": m_mc * t_mc, "extrapolated": True,
              "how": "eps-optimal cost (Eq. opt_M_ell, max over the quantities) from the timed steps' V_l "
                     "(level 0: 20000 samples apart) at the batch's cell-step rate; plain MC from "
                     "2 Var[P_L]/eps^2 samples at the measured MC time per sample of the finest level"}
    if learned is not None:
        pS, pC = acc_parts
        Vs = np.zeros((L + 2, nq))
        ts = [pS[0, 5] / pS[0, 0], pC[0, 5] / pC[0, 0]] + t_l[1:]
        for i, p in enumerate((pS, pC)):
            n = p[:, 0]
            Vs[i] = np.maximum(0.0, (p[:, 2] - p[:, 1] ** 2 / n) / (n - 1))
        Vs[2:] = V[1:]
        M_sur, t_sur = opt_cost(Vs, ts)
        sur.update({"var_P0": V[0].tolist(), "var_S": Vs[0].tolist(), "var_P0_minus_S": Vs[1].tolist(),
                    "s_per_sample_S": ts[0], "s_per_sample_P0_minus_S": ts[1], "s_per_sample_P0": t_l[0],
                    "M_opt": M_sur.tolist(), "mlmc_s_to_eps": t_sur,
                    "mlmc_s_to_eps_incl_training": t_sur + sur["train_s"], "extrapolated": True})

    extras = {}
    if not args.no_secondary:
        extras = secondary(args, stream)

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
            h2d_k = c2.level_info(0).h2d_bytes
            d2h_k = 8 * S * (L + 1) + 4
            if learned is not None:
                c2.surrogate_init(seed0 + 3)
                c2.surrogate_params(theta)            # the trained network: host -> device
                h2d_k += 4 * theta.size
            res = c2.run_batch(batch_counts, seed0 + 101 + k)      # host sums of every level
            if learned is not None:
                for part, n in ((-1, learned[0]), (0, learned[1])):
                    c2.run_surrogate(part, n, seed0 + 101 + k)
                    d2h_k += 8 * S + 4
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
               "what": "mlmc_dk_init (mean fields + pinned uploads) + the trained network's parameters + "
                       "mlmc_dk_run_batch (host sums) + mlmc_dk_run_surrogate (both parts) + free"}
        ctx = None

    if rank != 0:
        if ctx is not None:
            ctx.close()
        return None
    cpu, oerr = None, None
    if world == 1 and not args.no_cpu_baseline:
        # the oracle on a bounded sample of the step's own ids (seed of the first timed step),
        # which also gives the per-sample error of the GPU path on those ids
        cpu, outs = oracle_leg(wl, alloc, learned, args.cpu_budget, seed0 + 101, first0)
        c3 = ctx or mlmc_dk.Context.from_workload(wl, stream=stream.cuda_stream)
        oerr = oracle_error(c3, wl, outs, seed0 + 101, stream)
        summary = {"same_kernels_as": "oracle_error", "worst_err_over_bar_scale": oerr["worst_err_over_bar_scale"],
                   "within_bar": oerr["within_bar"]}
        to_eps["oracle_error"] = summary
        if sur is not None:
            c3.surrogate_init(seed0 + 3)
            c3.surrogate_params(theta)
            sur["oracle_error"] = dict(summary, network=network_error(c3, theta, c3.surrogate_info()[1],
                                                                      4096, seed0 + 23))
        c3.close()
        ctx = None
    if ctx is not None:
        ctx.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32 fixed-point state, f32 noise, f64 sums, bf16 network",
        "data": "synthetic",
        "config": dict(workload_config(wl, alloc, learned),
                       sample_steps_per_step=sample_steps, cell_steps_per_step=cell_steps,
                       l2="512 MiB buffer zeroed between timed steps, outside the step events",
                       parallelism=f"{world} rank(s), disjoint sample ids per rank",
                       kernels=[{"n": i.n, "band": bool(i.band), "bands": i.bands, "in_flight": i.in_flight,
                                 "C": i.lane_cols, "R": i.lane_rows, "cluster": i.cluster} for i in info],
                       tune_s=tune_s, tuned=not args.no_tune, t_scale=args.t_scale,
                       batch_split={"level": split_level, "fraction": split_frac, "tune_s": split_s}),
        "cell_steps_per_s": world * cell_steps * args.steps / (total_ms * 1e-3),
        "gpu_launches": launches,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "estimate": {"values": est.tolist(), "se": np.sqrt(var).tolist(), "oracle_error": oerr},
        "oracle_error": oerr,
    }
    line["mlmc_s_to_eps"] = t_mlmc
    line["mc_s_to_eps"] = m_mc * t_mc
    line["mlmc_speedup_vs_mc"] = m_mc * t_mc / t_mlmc
    line["to_eps"] = to_eps
    if sur:
        line["surrogate"] = sur
        line["mlmc_surrogate_s_to_eps"] = sur["mlmc_s_to_eps_incl_training"]
    line.update(extras)
    return line


def secondary(args, stream):
    """Secondary measurements: the 16^2..256^2 workload's batch (the previous
    headline) with a measured Algorithm 1 run, the 512^2 large-grid stencil,
    the theta-scheme and the Fourier-coupled kernels."""
    out = {}
    if not args.no_mlmc16:
        out["mlmc16_256"] = mlmc16_batch(args, stream)
    if not args.no_streamed:
        out["large_grid_stencil"] = streamed_stencil(stream)
    if not args.no_theta:
        out["theta_scheme"] = theta_scheme(stream)
    if not args.no_fourier:
        out["fourier_coupling"] = fourier_coupling(stream)
    return out


def mlmc16_batch(args, stream):
    """The 16^2..256^2 workload (N = 1e5, eps = 1e-3): its scaled eps-optimal
    batch timed over three steps, and a complete Algorithm 1 run at eps = 1e-2
    (levels added by the stopping test), both through the batch graph."""
    import torch
    from paper_2311_08872_gb300 import mlmc_dk, workloads
    wl = workloads.get("mlmc16_256")
    alloc = list(wl.alloc)
    with mlmc_dk.Context.from_workload(wl, stream=stream.cuda_stream) as c:
        c.tune(1)
        # batch split: a share of the 256^2 level's samples on the streamed kernels
        # beside its 8-CTA clusters (the SMs those cannot use)
        split_frac, split_s = c.tune_batch(alloc, 1)
        info = [c.level_info(l) for l in range(wl.L_max + 1)]
        steps = sum(m * i.M for m, i in zip(alloc, info))
        sums = torch.zeros(wl.L_max + 1, mlmc_dk.sums_len(c.n_quant), dtype=torch.float64, device="cuda")
        c.run_batch_dev(alloc, 0, 3, sums.data_ptr(), stream.cuda_stream)      # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(3):
            c.run_batch_dev(alloc, 1000 * (k + 1), 5 + k, sums.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        level_ms = c.batch_level_ms()
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = c.estimate(args.adaptive_eps, relative=True, seed=wl.seed + 5)
        torch.cuda.synchronize()
        adaptive = {"eps_rel": args.adaptive_eps, "s": time.perf_counter() - t, "L": r.L,
                    "M": [r.M[l] for l in range(r.L + 1)], "estimate": r.estimate, "variance": r.variance,
                    "eps_abs": r.eps_abs, "converged": bool(r.converged), "cell_steps": r.cell_steps}
        if not args.no_cpu_baseline:
            # the oracle on the first ids of the run's levels up to 128^2 (same seed)
            counts = [min(r.M[l], 8 if info[l].n <= 64 else 4) for l in range(min(r.L, 3) + 1)]
            outs = oracle_samples(wl, counts, wl.seed + 5)
            adaptive["oracle_error"] = oracle_error(c, wl, outs, wl.seed + 5, stream)
    fin = info[-1]
    return {"alloc": alloc, "ms_per_step": ms, "coupled_sample_steps_per_s": steps / (ms * 1e-3),
            "batch_split": {"fraction": split_frac, "tune_s": split_s},
            "cell_steps_per_s": sum(m * i.cost for m, i in zip(alloc, info)) / (ms * 1e-3),
            "level_ms": level_ms, "kernels": [{"n": i.n, "band": bool(i.band), "cluster": i.cluster} for i in info],
            "algorithm1_measured": adaptive,
            "closed_form_EP_finest": closed_form_EP_cos1(fin.n, fin.tau, fin.M)}


def run_reference(args, wl, rank, world):
    """The reference arm: the FP64 oracle (there is no published implementation)
    as it stands, on the host cores, on a bounded sample of the same workload
    and step allocation, scaled to the step by level."""
    if rank != 0:
        return None
    if wl.alloc is None:
        return {"impl": "reference", "unavailable": "workload has no fixed allocation"}
    alloc = list(wl.alloc) + [0] * (wl.L_max + 1 - len(wl.alloc))
    learned = tuple(wl.alloc_learned) if (wl.alloc_learned and not args.no_surrogate) else None
    M, fine, coarse = oracle_level_costs(wl)
    sample_steps, cell_steps = step_units(fine, coarse, M, alloc, learned)
    budget = max(2.0, args.cpu_budget / 3)
    for w in range(args.warmup):
        oracle_leg(wl, alloc, learned, budget / 2, wl.seed + 17 + w, 0)
    vals, res = [], None
    for k in range(args.steps):
        res, _ = oracle_leg(wl, alloc, learned, budget, wl.seed + 101 + k, 0)
        vals.append(res["batch_cpu_s"])
    cpu_s = statistics.mean(vals)
    value = sample_steps / cpu_s
    cb = dict(res)
    cb["value"] = value
    cfg = dict(workload_config(wl, alloc, learned), sample_steps_per_step=sample_steps,
               cell_steps_per_step=cell_steps,
               what="FP64 oracle (plain C) per coupled sample on the host cores; each step times a bounded sample "
                    "of the step's allocation and scales it to the full step by level (learned level: the "
                    "correction level's level-0 paths, network cost not counted)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * cpu_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def profile_level(spec):
    """One level batch, run twice (warm-up, then timed with CUDA events): the
    small, repeatable case behind the kernel profiles."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2311_08872_gb300 import mlmc_dk, workloads
    parts = spec.split(":")
    wl = workloads.get(parts[0])
    level, count = int(parts[1]), int(parts[2])
    if len(parts) > 3 and parts[3]:
        wl = wl.with_(T=float(parts[3]))
    st = torch.cuda.current_stream()
    with mlmc_dk.Context.from_workload(wl, stream=st.cuda_stream) as ctx:
        if len(parts) > 4:
            ctx.set_variant(level, level > 0, int(parts[4]))
        info = ctx.level_info(level)
        sums = torch.zeros(mlmc_dk.sums_len(ctx.n_quant), dtype=torch.float64, device="cuda")
        ctx.run_level_dev(level, 0, 0, count, wl.seed, sums.data_ptr(), 0, st.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctx.run_level_dev(level, 0, count, count, wl.seed, sums.data_ptr(), 0, st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    print(json.dumps({"workload": wl.name, "level": level, "n": info.n, "fine_steps": info.M, "samples": count,
                      "streamed": bool(info.streamed), "band": bool(info.band), "variant": info.variant_coupled,
                      "in_flight": info.in_flight, "ms": ms, "cell_steps_per_s": count * info.cost / (ms * 1e-3),
                      "fine_cell_steps_per_s": count * info.cost_mc / (ms * 1e-3)}))


def profile_gemm(rows):
    """The learned level's network forward (three 256-wide dense layers on the
    tensor cores, then the output layer) on `rows` random feature rows, run
    twice; the second run is timed with CUDA events."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2311_08872_gb300 import mlmc_dk, workloads
    wl = workloads.get("mlmc16_256").with_(L_max=1)
    X = np.random.default_rng(1).normal(size=(rows, 64)).astype(np.float32)
    with mlmc_dk.Context.from_workload(wl) as ctx:
        ctx.surrogate_init(1)
        ctx.surrogate_forward(X)
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx.surrogate_forward(X)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t
    flops = 2.0 * rows * (64 * 256 + 2 * 256 * 256)
    print(json.dumps({"rows": rows, "gemm_flops": flops, "forward_s_incl_copies": sec}))


def main():
    args = parse()
    if args.profile_level:
        profile_level(args.profile_level)
        return
    if args.profile_gemm:
        profile_gemm(args.profile_gemm)
        return
    from paper_2311_08872_gb300 import workloads
    wl = workloads.get(args.workload)
    if args.t_scale != 1.0:
        wl = wl.with_(T=wl.T / args.t_scale)
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
