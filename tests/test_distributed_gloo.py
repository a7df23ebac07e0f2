"""Multi-rank host logic on CPU: two gloo ranks shard sample ids, all-reduce
their FP64 level sums (max for the mass error) and time by the slowest rank."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2311_08872_gb300 import distributed as D

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sums = np.zeros((3, 14))
        sums[:, 0] = 10 + rank                       # sample counts
        sums[:, 1] = [0.0, 1e-12 * rank, 0.0]        # mass error: maximum
        sums[:, 2:] = np.arange(12) * (rank + 1)
        red = D.allreduce_sums(sums)
        t = D.max_over_ranks(1.0 + rank)
        out.put((rank, red, t, D.first_sample(rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_level_sums():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, red, t, first in res:
        assert np.all(red[:, 0] == 21)
        assert red[1, 1] == 1e-12 and red[0, 1] == 0.0
        np.testing.assert_array_equal(red[:, 2:], np.tile(np.arange(12) * 3.0, (3, 1)))
        assert t == 2.0
        assert first == rank * (1 << 40)
    from paper_2311_08872_gb300.distributed import weak_scaling_value
    assert weak_scaling_value(100.0, 2.0, 2) == 100.0


# ---------------------------------------------------------- Algorithm 1 across ranks
def _oracle_sampler(wl):
    """run_level(level, first, count) -> sums in the device layout, from the
    FP64 oracle (stands in for the GPU path of each rank)."""
    import oracle
    levels = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu, wl.M0, ratio=wl.ratio)
    rho0, phi = wl.rho0_all(), wl.phi_all()
    ybar = [oracle.inner_h(oracle.mean_field(l.n, l.h, l.tau, l.M, rho0[l.level]), phi[l.level][0], l.h)
            for l in levels]
    cost = [levels[l].n ** 2 * levels[l].M + (levels[l - 1].n ** 2 * levels[l - 1].M if l else 0)
            for l in range(len(levels))]

    def run_level(l, first, count):
        ol = oracle.level_inputs(wl.length, levels, wl.N, rho0, phi, l, l > 0, coupling=wl.coupling)
        r = oracle.run_samples(ol, wl.seed, range(first, first + count), l > 0)
        df = r["Y_f"][:, 0] - ybar[l]
        dc = r["Y_c"][:, 0] - ybar[l - 1] if l else np.zeros(count)
        pf, pc = wl.N * df ** 2, (wl.N * dc ** 2 if l else np.zeros(count))
        dp = pf - pc
        return np.array([count, 0.0, dp.sum(), (dp ** 2).sum(), (dp ** 3).sum(), (dp ** 4).sum(),
                         pf.sum(), (pf ** 2).sum(), pc.sum(), (pc ** 2).sum(), df.sum(), (df ** 2).sum(),
                         dc.sum(), (dc ** 2).sum()])
    return run_level, cost


def _small_workload(fourier=False):
    from paper_2311_08872_gb300 import workloads as W
    if fourier:
        return W.get("fourier6_54").with_(L_max=1)
    return W.get("mlmc16_256").with_(n0=8, L_max=3, T=0.005, N=1e5)


def _estimate_worker(rank, world, port, out, fourier=False):
    import torch.distributed as dist
    from paper_2311_08872_gb300 import distributed as D
    from paper_2311_08872_gb300 import mlmc_dk

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = _small_workload(fourier)
        run_level, cost = _oracle_sampler(wl)
        r = D.estimate(run_level, wl.L_max, 0.03, cost, 14, ratio=float(wl.ratio), pilot=64, world=world,
                       rank=rank, reduce=D.allreduce_sums)
        out.put((rank, r["estimate"], r["variance"], r["L"], r["M"], r["converged"]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("fourier", [False, True])
def test_algorithm1_across_two_gloo_ranks_matches_one_rank(fourier):
    """Two ranks share every round's new sample ids and all-reduce the level
    sums; they take the same decisions as one rank running all the ids (NN
    hierarchy, and the Fourier coupling's ratio-3 hierarchy)."""
    import multiprocessing as mp
    from paper_2311_08872_gb300 import distributed as D

    wl = _small_workload(fourier)
    run_level, cost = _oracle_sampler(wl)
    ref = D.estimate(run_level, wl.L_max, 0.03, cost, 14, ratio=float(wl.ratio), pilot=64)
    assert ref["converged"] or ref["L"] == wl.L_max
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_estimate_worker, args=(r, 2, port, q, fourier)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, est, var, L, M, conv in res:
        assert L == ref["L"] and M == ref["M"] and conv == ref["converged"]
        assert est == pytest.approx(ref["estimate"], rel=1e-12)
        assert var == pytest.approx(ref["variance"], rel=1e-10)
