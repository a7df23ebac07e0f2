"""Multi-level batch (all levels concurrently, captured in a CUDA graph):
identical samples and sums to the per-level launches, graph reuse across
parameter changes and re-instantiation across shape changes."""
import numpy as np
import pytest

from paper_2311_08872_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2311_08872_gb300 import build as libbuild
    libbuild.build()
    from paper_2311_08872_gb300 import mlmc_dk
    return mlmc_dk


def test_batch_equals_per_level_launches(dk):
    import torch
    wl = W.get("mlmc16_256").with_(L_max=3)
    st = torch.cuda.current_stream().cuda_stream
    with dk.Context.from_workload(wl) as ctx:
        S = dk.sums_len(ctx.n_quant)
        for counts, first, seed in (([3000, 400, 60, 12], 0, 5), ([3000, 400, 60, 12], 77, 6),
                                    ([1000, 0, 30, 4], 5, 7)):
            batch = torch.full((4, S), float("nan"), dtype=torch.float64, device="cuda")
            ctx.run_batch_dev(counts, first, seed, batch.data_ptr(), st)
            torch.cuda.synchronize()
            ms = ctx.batch_level_ms()
            for l, m in enumerate(counts):
                ref = torch.zeros(S, dtype=torch.float64, device="cuda")
                ctx.run_level_dev(l, 0, first, m, seed, ref.data_ptr(), 0, st)
                torch.cuda.synchronize()
                np.testing.assert_allclose(batch[l].cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=0)
                if m > 0:
                    assert ms[l] > 0


def test_host_batch_matches_host_levels(dk):
    wl = W.get("mlmc16_256").with_(L_max=2)
    counts = [2000, 300, 40]
    with dk.Context.from_workload(wl) as a, dk.Context.from_workload(wl) as b:
        got = a.run_batch(counts, seed=9)
        for l, m in enumerate(counts):
            ref = b.run_level(l, m, seed=9)
            for q in range(a.n_quant):
                g, r = got[l][q], ref[q]
                assert g.n == r.n == m
                for k in ("dp1", "dp2", "dp3", "dp4", "pf1", "pf2", "pc1", "pc2", "yf1", "yf2", "yc1", "yc2"):
                    assert getattr(g, k) == pytest.approx(getattr(r, k), rel=1e-12, abs=0)
        assert [a.level_info(l).next_sample for l in range(3)] == counts
