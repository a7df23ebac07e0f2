"""Band kernels: a sample of a large grid spread over several CTAs (full-width
bands of coarse rows held in registers, band edges exchanged through global
memory with per-step counters, cooperative launch).

* On 128^2 and 256^2 levels they reproduce the register kernels and on 512^2
  and 1024^2 levels the streamed-state kernels: identical fixed-point paths
  (equal masses), observables equal up to summation order.
* Several waves of samples in flight, ragged last waves, the plain-MC stream.
* Oracle parity at 512^2 and 1024^2 runs through them (tests/test_gpu_stream.py:
  the band kernel is the default on those levels).
"""
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


def _samples(ctx, dk, level, tag, first, count, seed):
    import torch
    sums = torch.zeros(dk.sums_len(ctx.n_quant), dtype=torch.float64, device="cuda")
    samp = torch.zeros(count, dk.sample_stride(ctx.n_obs), dtype=torch.float64, device="cuda")
    ctx.run_level_dev(level, tag, first, count, seed, sums.data_ptr(), samp.data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return sums.cpu().numpy(), samp.cpu().numpy()


def _band_variants(ctx, level):
    """Indices of the band-kernel builds among the level's variants (the last
    ones: 4 x 8 thread blocks where the grid allows them, then 4 x 4)."""
    n = ctx.level_info(level).n_variants
    return [v for v in range(n) if v >= n - (2 if ctx.level_info(level).n >= 256 else 1)]


def _band_variant(ctx, level, coupled, v=None):
    """Select a band-kernel build (default: the last variant) for the level's
    coupled or fine-only kernel; level_info describes the coupled kernel of a
    level >= 1."""
    ctx.set_variant(level, coupled, ctx.level_info(level).n_variants - 1 if v is None else v)
    d = ctx.level_info(level)
    if coupled or level == 0:
        assert d.band == 1 and d.bands >= 2 and d.in_flight >= 1
    return d


def _compare(a, b, K, tol):
    assert np.array_equal(a[:, 2 * K:], b[:, 2 * K:])            # masses: same integer paths
    scale = np.sqrt(np.mean(a[:, :2 * K] ** 2, axis=0)) + 1e-300
    err = np.abs(a[:, :2 * K] - b[:, :2 * K]) / scale
    assert np.all(err <= tol), float(err.max())


@pytest.mark.parametrize("level,count", [(3, 40), (4, 23)])
def test_band_equals_register_kernels(dk, level, count):
    """128^2 / 256^2 (with 64^2 / 128^2 coarse): more samples than one wave
    in flight on 128^2, a ragged count on both."""
    wl = W.get("mlmc16_256").with_(L_max=level, T=0.002)
    with dk.Context.from_workload(wl) as reg, dk.Context.from_workload(wl) as bnd:
        for v in _band_variants(bnd, level):
            for tag in (0, 1):
                coupled = tag == 0
                d = _band_variant(bnd, level, coupled, v)
                s_r, a = _samples(reg, dk, level, tag, 3, count, 11)
                s_b, b = _samples(bnd, dk, level, tag, 3, count, 11)
                _compare(a, b, reg.n_obs, 1e-6)
                assert s_b[0] == count and s_b[1] == 0.0
                print(level, v, tag, "bands", d.bands, "in flight", d.in_flight)


def test_band_many_waves(dk):
    """More than two waves of 256^2 samples in flight, the last one ragged,
    against the streamed-state kernels forced onto the same level: both project
    the integer states on FP64 test functions in FP64, so identical paths give
    observables equal to FP64 summation order."""
    wl = W.get("mlmc16_256").with_(L_max=4, T=2.5e-4)
    with dk.Context.from_workload(wl, stream_from_n=256) as stm, dk.Context.from_workload(wl) as bnd:
        for v in _band_variants(bnd, 4):
            d = _band_variant(bnd, 4, True, v)
            count = 2 * d.in_flight + 5
            _, a = _samples(stm, dk, 4, 0, 100, count, 7)
            s, b = _samples(bnd, dk, 4, 0, 100, count, 7)
            _compare(a, b, bnd.n_obs, 1e-10)
            assert s[0] == count


def test_band_256_matches_oracle(dk):
    """The band kernel on the benchmark workload's 256^2 level (coupled with
    128^2) over 1536 fine steps, sample by sample against the FP64 oracle."""
    import oracle
    wl = W.get("mlmc16_256").with_(T=0.0025)
    with dk.Context.from_workload(wl) as ctx:
        _band_variant(ctx, 4, True)
        info = ctx.level_info(4)
        _, samp = _samples(ctx, dk, 4, 0, 40, 4, 13)
    lv = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu)
    ol = oracle.level_inputs(wl.length, lv, wl.N, wl.rho0_all(), wl.phi_all(), 4, True)
    ref = oracle.run_samples(ol, 13, range(40, 44), True, processes=4)
    for col, key, yb in ((0, "Y_f", info.ybar_f[0]), (1, "Y_c", info.ybar_c[0])):
        y = samp[:, col] + yb
        yo = ref[key][:, 0]
        rms = np.sqrt(np.mean((yo - yb) ** 2))
        assert np.all(np.abs(y - yo) <= 1e-5 * np.maximum(np.abs(yo), rms)), (key, y - yo, rms)


@pytest.mark.parametrize("name,kw,level,count", [
    ("lowdens32_512", dict(n0=256, L_max=1, T=4.0e-6), 1, 6),
    ("large32_1024", dict(n0=512, L_max=1, T=1.52e-6), 1, 3),
])
def test_band_equals_streamed_kernels(dk, name, kw, level, count):
    wl = W.get(name).with_(**kw)
    with dk.Context.from_workload(wl) as ctx:
        d = ctx.level_info(level)
        assert d.streamed == 1 and d.n_variants == 8 and d.band == 0      # the streamed kernel is the default
        for tag in (0, 1):
            coupled = tag == 0
            ctx.set_variant(level, coupled, 0)
            _, a = _samples(ctx, dk, level, tag, 2, count, 5)
            for v in _band_variants(ctx, level):
                _band_variant(ctx, level, coupled, v)
                _, b = _samples(ctx, dk, level, tag, 2, count, 5)
                _compare(a, b, ctx.n_obs, 1e-9)


def test_band_kernels_are_tuner_candidates_on_large_levels(dk):
    wl = W.get("large32_1024")
    with dk.Context.from_workload(wl) as ctx:
        for level in (3, 4, 5):
            d = ctx.level_info(level)
            # 256^2: two register builds; 512^2, 1024^2: six streamed builds; then two band builds
            assert d.band == 0 and d.n_variants == (4 if level == 3 else 8)
        secs = ctx.tune(1)
        assert secs > 0
        print("variants after tuning", ctx.variants())


def test_batch_with_band_level(dk):
    """A multi-level batch whose finest level runs on the band kernel (beside
    the graph of the register levels): the same sums as per-level launches."""
    import torch
    wl = W.get("mlmc16_256").with_(T=0.004)
    st = torch.cuda.current_stream().cuda_stream
    counts = [3000, 400, 60, 30, 25]
    with dk.Context.from_workload(wl) as ctx:
        _band_variant(ctx, 4, True)
        S = dk.sums_len(ctx.n_quant)
        batch = torch.full((5, S), float("nan"), dtype=torch.float64, device="cuda")
        ctx.run_batch_dev(counts, 4, 12, batch.data_ptr(), st)
        torch.cuda.synchronize()
        ms = ctx.batch_level_ms()
        assert ms[4] > 0 and ctx.level_info(4).batch_streamed == 0
        for l, m in enumerate(counts):
            ref = torch.zeros(S, dtype=torch.float64, device="cuda")
            ctx.run_level_dev(l, 0, 4, m, 12, ref.data_ptr(), 0, st)
            torch.cuda.synchronize()
            np.testing.assert_allclose(batch[l].cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=0)


def test_band_bounded_wait_reports_timeout(dk):
    """Failure detection without a fault: one band never publishes its edges,
    its neighbours' waits (limited to 4096 polls) run out, the kernel records
    the timeout and stops, the call returns MLMC_DK_ERR_TIMEOUT, and the same
    context then runs correct samples."""
    wl = W.get("mlmc16_256").with_(L_max=4, T=2.5e-4)
    with dk.Context.from_workload(wl) as ctx, dk.Context.from_workload(wl, stream_from_n=256) as stm:
        _band_variant(ctx, 4, True)
        assert ctx.band_wait_test(4, 4096, 1) == dk.ERR_TIMEOUT
        _, a = _samples(stm, dk, 4, 0, 0, 3, 9)
        s, b = _samples(ctx, dk, 4, 0, 0, 3, 9)
        _compare(a, b, ctx.n_obs, 1e-10)
        assert s[0] == 3
