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


@pytest.mark.parametrize("persistent", [False, True])
def test_batch_with_streamed_levels_beside_the_graph(dk, persistent):
    """The four-mode workload's 512^2 and 1024^2 levels run on the streamed
    kernels on their own streams beside the graph of the register levels
    (short horizon): the same sums as per-level launches, with one launch per
    step or the persistent launch on the streamed levels."""
    import torch
    wl = W.get("large32_1024").with_(T=1e-6)
    st = torch.cuda.current_stream().cuda_stream
    counts = [300, 60, 12, 5, 4, 3]
    with dk.Context.from_workload(wl) as ctx:
        if persistent:
            for l in (4, 5):
                ctx.set_variant(l, True, 3)
                assert ctx.level_info(l).persistent == 1
        assert ctx.level_info(4).streamed == 1 and ctx.level_info(5).streamed == 1
        S = dk.sums_len(ctx.n_quant)
        batch = torch.full((6, S), float("nan"), dtype=torch.float64, device="cuda")
        ctx.run_batch_dev(counts, 9, 21, batch.data_ptr(), st)
        torch.cuda.synchronize()
        ms = ctx.batch_level_ms()
        for l, m in enumerate(counts):
            ref = torch.zeros(S, dtype=torch.float64, device="cuda")
            ctx.run_level_dev(l, 0, 9, m, 21, ref.data_ptr(), 0, st)
            torch.cuda.synchronize()
            np.testing.assert_allclose(batch[l].cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=0)
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


def _close(a, b, tol=1e-5):
    """Level sums of the same samples from two kernel families: counts and the
    mass-error maximum equal; the k-th power sums of a quantity x agree to tol
    times (sum x^2)^(k/2), a bound on sum |x|^k (FP32 partial-sum order of the
    observables differs between the families)."""
    assert a[0] == b[0] and a[1] == b[1]
    q = (len(a) - 2) // 12
    for i in range(q):
        s = a[2 + 12 * i: 2 + 12 * (i + 1)]
        t = b[2 + 12 * i: 2 + 12 * (i + 1)]
        dp2, pf2, pc2, yf2, yc2 = abs(s[1]), abs(s[5]), abs(s[7]), abs(s[9]), abs(s[11])
        n = a[0]
        bound = [np.sqrt(n * dp2), dp2, dp2 ** 1.5, dp2 ** 2, np.sqrt(n * pf2), pf2, np.sqrt(n * pc2), pc2,
                 np.sqrt(n * yf2), yf2, np.sqrt(n * yc2), yc2]
        for j in range(12):
            assert abs(s[j] - t[j]) <= tol * bound[j] + 1e-300, (i, j, s[j], t[j], bound[j])


def test_batch_split_runs_the_same_samples(dk):
    """Part of the 256^2 level's samples on the streamed kernels beside the
    graph: same sample ids and paths, so the level's sums match the unsplit
    batch; the other levels' sums are untouched bit for bit."""
    import torch
    wl = W.get("mlmc16_256")
    st = torch.cuda.current_stream().cuda_stream
    counts = [4000, 400, 60, 10, 9]
    with dk.Context.from_workload(wl) as ctx:
        S = dk.sums_len(ctx.n_quant)
        info = ctx.level_info(4)
        assert info.split_capable == 1 and ctx.level_info(3).split_capable == 0
        with pytest.raises(dk.MLMCError):
            ctx.set_batch_split(3, 0.1)
        ref = torch.zeros((5, S), dtype=torch.float64, device="cuda")
        ctx.run_batch_dev(counts, 3, 8, ref.data_ptr(), st)
        torch.cuda.synchronize()
        assert ctx.level_info(4).batch_streamed == 0
        ctx.set_batch_split(4, 0.5)
        for rep in range(2):
            got = torch.full((5, S), float("nan"), dtype=torch.float64, device="cuda")
            ctx.run_batch_dev(counts, 3, 8, got.data_ptr(), st)
            torch.cuda.synchronize()
            assert ctx.level_info(4).batch_streamed == 4
            g, r = got.cpu().numpy(), ref.cpu().numpy()
            np.testing.assert_array_equal(g[:4], r[:4])
            _close(g[4], r[4])
        f, secs = ctx.tune_batch(counts, 1)
        assert f in (0.0, 0.04, 0.06, 0.08, 0.10, 0.12) and secs > 0
        assert ctx.level_info(4).split_fraction == f
