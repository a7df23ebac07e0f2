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
