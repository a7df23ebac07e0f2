"""Multi-rank helpers (one process per GPU, torch.distributed for plumbing).

Samples are independent and a pure function of (seed, level, stream, id), so
ranks shard by sample ids: rank r of R takes ids r * span + [0, count).  The
only exchange an Algorithm 1 across ranks needs is the per-level FP64 moment
sums once per iteration: a sum all-reduce, with the maximum for the
mass-error entry (index 1 of the device sums layout).
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
