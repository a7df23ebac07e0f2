"""Multi-rank helpers (one process per GPU, torch.distributed for plumbing).

Samples are independent and a pure function of (seed, level, stream, id), so
ranks shard by sample ids: in the benchmark rank r of R takes ids
r * span + [0, count); Algorithm 1 across ranks (`estimate`) splits each
round's new ids of a level into R contiguous pieces.  The only exchange an
Algorithm 1 across ranks needs is the per-level FP64 moment sums once per
iteration: a sum all-reduce, with the maximum for the mass-error entry
(index 1 of the device sums layout).  Every rank then takes the same
decisions from the same global sums, so no broadcast is needed.
"""
from __future__ import annotations

import numpy as np

ID_SPAN = 1 << 40   # sample ids per rank (the 48-bit id space holds 256 ranks)


def first_sample(rank: int, span: int = ID_SPAN) -> int:
    return rank * span


def allreduce_sums(sums: np.ndarray, group=None) -> np.ndarray:
    """sums: float64 [..., 2 + n_quant * 12] in the layout of mlmc_dk_run_level_dev."""
    import torch
    import torch.distributed as dist

    t = torch.from_numpy(np.ascontiguousarray(sums, dtype=np.float64)).clone()
    mx = t[..., 1].clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX, group=group)
    t[..., 1] = mx
    return t.numpy()


def max_over_ranks(x: float, group=None) -> float:
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def weak_scaling_value(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds_max


def merge_sums(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Sums of two disjoint sample sets of the same levels (index 1: max)."""
    out = a + b
    out[..., 1] = np.maximum(a[..., 1], b[..., 1])
    return out


def estimate(run_level, L_max: int, eps: float, cost, width: int, *, ratio: float = 2.0, relative: bool = True,
             pilot: int = 256, L_start: int = 2, world: int = 1, rank: int = 0, reduce=None):
    """Algorithm 1 (Section 7.1) with the samples of every round shared by the
    ranks: the library's mlmc_dk_algorithm1 drives it (targets, stopping test
    and estimator are computed there, identically on every rank).

    run_level(level, first_id, count) -> this rank's sums of `count` coupled
    samples with ids first_id.. (float64 [width], the device sums layout,
    width = 2 + 12 n_quant); cost[l]: cost of one sample of level l; ratio:
    the hierarchy's mesh ratio (2 NN, 3 Fourier); reduce(local) -> global sums
    over ranks (allreduce_sums; required when world > 1).  The union over the
    ranks of each round's pieces is the id range a single rank would run, so
    decisions and estimate do not depend on the number of ranks (up to FP64
    summation order).  Returns the estimate, its variance, L, samples per
    level, eps_abs and convergence."""
    from . import mlmc_dk

    n_quant = (width - 2) // mlmc_dk.NSUM

    def run_round(L, first, count):
        out = np.zeros((L_max + 1, width))
        for l in range(L_max + 1):
            if count[l] > 0:
                out[l] = run_level(l, first[l], count[l])
        return out

    r = mlmc_dk.algorithm1(run_round, reduce, L_max, n_quant, cost, eps, ratio=ratio, relative=relative,
                           pilot=pilot, L_start=L_start, rank=rank, world=world)
    return {"estimate": r.estimate, "variance": r.variance, "L": r.L, "M": [int(r.M[l]) for l in range(r.L + 1)],
            "eps_abs": r.eps_abs, "converged": bool(r.converged)}
