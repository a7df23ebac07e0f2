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


def estimate(run_level, L_max: int, eps: float, cost, plan, width: int, *, relative: bool = True,
             pilot: int = 256, L_start: int = 2, world: int = 1, rank: int = 0, reduce=None,
             max_iter: int = 1000):
    """Algorithm 1 (Section 7.1) with the samples of every round shared by the ranks.

    run_level(level, first_id, count) -> this rank's sums of `count` coupled
    samples with ids first_id.. (float64 [width], the device sums layout,
    width = 2 + 12 n_quant); cost[l]: cost of one sample of level l;
    plan(n, s1, s2, cost, eps_abs) -> (targets, converged): the host step of
    Eq. (opt_M_ell) and Eq. (convergence_criterion) (mlmc_dk.plan);
    reduce(local) -> global sums over ranks (allreduce_sums; unused on one
    rank).  Each round the missing samples of level l, ids next[l] ..
    target[l]-1, are cut into `world` contiguous pieces and piece `rank` runs
    here; the union over ranks is the id range a single rank would run, so
    decisions and estimate do not depend on the number of ranks (up to FP64
    summation order).  The first quantity drives the allocation; eps is
    relative to the pilot estimate when `relative` (frozen after the pilot).
    Returns the estimate, its variance, L, samples per level, eps_abs,
    convergence and the per-level global sums.
    """
    if pilot <= 0:
        raise ValueError("pilot must be positive")
    L = min(L_start, L_max)
    sums = np.zeros((L_max + 1, width))
    nxt = [0] * (L_max + 1)
    target = [pilot if l <= L else 0 for l in range(L_max + 1)]
    eps_abs = None if relative else eps
    converged = False
    for _ in range(max_iter):
        rnd = np.zeros((L_max + 1, width))
        for l in range(L + 1):
            need = target[l] - nxt[l]
            if need <= 0:
                continue
            base, extra = divmod(need, world)
            cnt = base + (1 if rank < extra else 0)
            if cnt > 0:
                rnd[l] = run_level(l, nxt[l] + rank * base + min(rank, extra), cnt)
            nxt[l] += need
        if reduce is not None and world > 1:
            rnd = reduce(rnd)
        sums = merge_sums(sums, rnd)
        n = [int(round(sums[l, 0])) for l in range(L + 1)]
        s1 = [float(sums[l, 2]) for l in range(L + 1)]
        s2 = [float(sums[l, 3]) for l in range(L + 1)]
        if eps_abs is None:
            eps_abs = eps * abs(sum(a / b for a, b in zip(s1, n)))
            if not eps_abs > 0:
                raise ValueError("relative eps with a zero pilot estimate")
        tgt, conv = plan(n, s1, s2, list(cost[:L + 1]), eps_abs)
        more = False
        for l in range(L + 1):
            target[l] = max(target[l], int(tgt[l]))
            if target[l] - n[l] > 0.01 * n[l]:
                more = True
        if more:
            continue
        if conv:
            converged = True
            break
        if L == L_max:
            break
        L += 1
        target[L] = pilot
    n = sums[:L + 1, 0]
    est = float(np.sum(sums[:L + 1, 2] / n))
    var = float(np.sum((sums[:L + 1, 3] - sums[:L + 1, 2] ** 2 / n) / (n - 1) / n))
    return {"estimate": est, "variance": var, "L": L, "M": [int(x) for x in n], "eps_abs": eps_abs,
            "converged": converged, "sums": sums[:L + 1]}
