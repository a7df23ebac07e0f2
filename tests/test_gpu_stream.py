"""Streamed-state kernels (grids too large for registers: 512^2, 1024^2).

* Forced onto 128^2 and 256^2 levels they must reproduce the register kernels:
  identical fixed-point paths (equal masses), observables equal up to the
  order of FP32 partial sums.
* At 512^2 (short horizon, so the oracle is affordable) they match the FP64
  oracle sample by sample.
* At the full 512^2 and 1024^2 levels of the low-density and large workloads:
  exact mass conservation, and with the noise off the observables equal the
  discrete mean field (a property that holds at any size).
"""
import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("level,count", [(3, 12), (4, 10)])
def test_streamed_equals_register_kernels(dk, level, count):
    wl = W.get("mlmc16_256").with_(L_max=level)
    with dk.Context.from_workload(wl) as reg, dk.Context.from_workload(wl, stream_from_n=128) as stm:
        assert stm.level_info(level).streamed == 1 and reg.level_info(level).streamed == 0
        for tag in (0, 1):
            s_r, a = _samples(reg, dk, level, tag, 3, count, 11)
            s_s, b = _samples(stm, dk, level, tag, 3, count, 11)
            K = reg.n_obs
            assert np.array_equal(a[:, 2 * K:], b[:, 2 * K:])
            scale = np.sqrt(np.mean(a[:, :2 * K] ** 2, axis=0)) + 1e-300
            assert np.all(np.abs(a[:, :2 * K] - b[:, :2 * K]) <= 1e-6 * scale)
            assert s_s[0] == count and s_s[1] == 0.0
            # power sums of signed terms cancel: compare against the sums of |terms|
            Df, Dc = a[:, :K], a[:, K:2 * K]
            pf = wl.N * Df[:, 0] ** 2
            pc = wl.N * Dc[:, 0] ** 2 if tag == 0 else np.zeros_like(pf)
            dp = np.abs(pf - pc)
            mag = np.array([dp.sum(), (dp ** 2).sum(), (dp ** 3).sum(), (dp ** 4).sum(), pf.sum(), (pf ** 2).sum(),
                            pc.sum(), (pc ** 2).sum(), np.abs(Df[:, 0]).sum(), (Df[:, 0] ** 2).sum(),
                            np.abs(Dc[:, 0]).sum(), (Dc[:, 0] ** 2).sum()])
            assert np.all(np.abs(s_s[2:] - s_r[2:]) <= 1e-5 * mag + 1e-300)


def test_streamed_512_matches_oracle(dk):
    # 256^2 / 512^2 levels over a short horizon: 2 and 8 fine steps
    wl = W.get("lowdens32_512").with_(n0=256, L_max=1, T=2.0e-6)
    with dk.Context.from_workload(wl) as ctx:
        info = ctx.level_info(1)
        assert info.n == 512 and info.streamed == 1 and info.M == 8
        _, samp = _samples(ctx, dk, 1, 0, 0, 3, 21)
    lv = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu)
    ol = oracle.level_inputs(wl.length, lv, wl.N, wl.rho0_all(), wl.phi_all(), 1, True)
    ref = oracle.run_samples(ol, 21, range(3), True)
    for col, key, yb in ((0, "Y_f", info.ybar_f[0]), (1, "Y_c", info.ybar_c[0])):
        y = samp[:, col] + yb
        yo = ref[key][:, 0]
        rms = np.sqrt(np.mean((yo - yb) ** 2))
        assert np.all(np.abs(y - yo) <= 1e-5 * np.maximum(np.abs(yo), rms)), (key, y - yo, rms)


def test_streamed_1024_four_modes_match_oracle(dk):
    """The largest grid (1024^2 fine, 512^2 coarse) of the four-mode workload
    over a short horizon (8 and 2 steps), four observables: sample by sample
    against the FP64 oracle."""
    wl = W.get("large32_1024").with_(n0=512, L_max=1, T=7.6e-7)
    with dk.Context.from_workload(wl) as ctx:
        info = ctx.level_info(1)
        assert info.n == 1024 and info.streamed == 1 and info.M == 8
        _, samp = _samples(ctx, dk, 1, 0, 5, 2, 33)
    lv = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu)
    ol = oracle.level_inputs(wl.length, lv, wl.N, wl.rho0_all(), wl.phi_all(), 1, True)
    ref = oracle.run_samples(ol, 33, range(5, 7), True)
    K = 4
    for k in range(K):
        for col, key, yb in ((k, "Y_f", info.ybar_f[k]), (K + k, "Y_c", info.ybar_c[k])):
            y = samp[:, col] + yb
            yo = ref[key][:, k]
            rms = np.sqrt(np.mean((yo - yb) ** 2))
            assert np.all(np.abs(y - yo) <= 1e-5 * np.maximum(np.abs(yo), rms)), (k, key, y - yo, rms)


@pytest.mark.parametrize("name,level,count", [("lowdens32_512", 4, 9), ("large32_1024", 5, 2)])
def test_full_size_streamed_levels_conserve_mass(dk, name, level, count):
    wl = W.get(name)
    with dk.Context.from_workload(wl) as ctx:
        info = ctx.level_info(level)
        assert info.streamed == 1
        sums, samp = _samples(ctx, dk, level, 0, 0, count, 5)
    assert sums[0] == count and sums[1] == 0.0
    assert np.all(np.isfinite(samp))


def test_full_size_1024_noise_off_is_mean_field(dk):
    wl = W.get("large32_1024").with_(N=0.0)
    with dk.Context.from_workload(wl) as ctx:
        sums, samp = _samples(ctx, dk, 5, 0, 0, 1, 5)
    K = 4
    # Y - Ybar: fixed-point rounding of a deterministic run only.  Each step rounds
    # every edge flux to within half a unit (2^-S); even fully coherent rounding
    # reaches (rho, phi)_h through grad phi only: <= 0.5 2^-S h^3 (2 n^2) 2 pi k per step,
    # about 5e-5 over the 524288 steps of 1024^2 (S = 26).
    assert np.all(np.abs(samp[:, :2 * K]) < 1e-4)
    print("max |Y - Ybar| with the noise off:", np.abs(samp[:, :2 * K]).max())
    assert sums[1] == 0.0


@pytest.mark.parametrize("name,kw,level,count", [
    ("lowdens32_512", dict(n0=256, L_max=1, T=2.0e-6), 1, 5),
    ("mlmc16_256", dict(L_max=4), 4, 3),
])
def test_streamed_kernel_variants_agree(dk, name, kw, level, count):
    """The six streamed variants (one launch per step, one persistent launch
    per wave, or one programmatic dependent launch per step; 4 or 5 resident
    CTAs per SM) compute the same integer paths and reduce them with the same
    observation kernel: outputs equal exactly; the tuner keeps one of them."""
    wl = W.get(name).with_(**kw)
    with dk.Context.from_workload(wl, stream_from_n=256) as ctx:
        info = ctx.level_info(level)
        assert info.streamed == 1 and info.n_variants == 6
        for tag in (0, 1):
            coupled = tag == 0
            outs = []
            for v in range(info.n_variants):
                ctx.set_variant(level, coupled, v)
                if coupled:   # level_info describes the coupled kernel of a level >= 1
                    d = ctx.level_info(level)
                    assert d.tile_rows == 32 and d.variant_coupled == v and d.persistent == (v in (2, 3))
                outs.append(_samples(ctx, dk, level, tag, 7, count, 4))
            for o in outs[1:]:
                assert np.array_equal(outs[0][1], o[1])
                assert np.array_equal(outs[0][0], o[0])
        secs = ctx.tune(1)
        assert secs > 0
        d = ctx.level_info(level)
        assert d.tile_rows == 32 and d.in_flight >= 1


def _persistent(ctx, level, coupled):
    """Select the persistent streamed build with 5 CTAs per SM (variant 3)."""
    ctx.set_variant(level, coupled, 3)
    d = ctx.level_info(level)
    if coupled or level == 0:
        assert d.persistent == 1 and d.streamed == 1
    return d


@pytest.mark.parametrize("name,kw,level", [
    ("lowdens32_512", dict(n0=256, L_max=1, T=4.0e-6), 1),
    ("large32_1024", dict(n0=512, L_max=1, T=1.52e-6), 1),
])
def test_persistent_waves_equal_per_step_launches(dk, name, kw, level):
    """Several waves of samples in flight and a ragged last wave through the
    persistent launch (CTAs take (tile, step) items from a counter and wait
    for the items they read from) give the same integer paths and the same
    outputs, bit for bit, as one launch per step; coupled and fine-only."""
    wl = W.get(name).with_(**kw)
    with dk.Context.from_workload(wl) as ctx:
        for tag in (0, 1):
            coupled = tag == 0
            d = _persistent(ctx, level, True)
            count = 2 * d.in_flight + 3
            _persistent(ctx, level, coupled)
            s_p, a = _samples(ctx, dk, level, tag, 11, count, 19)
            ctx.set_variant(level, coupled, 0)
            s_l, b = _samples(ctx, dk, level, tag, 11, count, 19)
            assert np.array_equal(a, b)
            assert s_p[0] == count and s_p[1] == 0.0
            np.testing.assert_allclose(s_p, s_l, rtol=1e-12, atol=0)


def test_persistent_and_pdl_full_size_1024_match_per_step_launches(dk):
    """The full 1024^2 level of the four-mode workload (524288 fine steps),
    two samples: the persistent launch and the programmatic dependent launches
    reproduce one launch per step exactly and conserve mass."""
    wl = W.get("large32_1024")
    with dk.Context.from_workload(wl) as ctx:
        _persistent(ctx, 5, True)
        s_p, a = _samples(ctx, dk, 5, 0, 0, 2, 5)
        ctx.set_variant(5, True, 5)
        s_d, c = _samples(ctx, dk, 5, 0, 0, 2, 5)
        ctx.set_variant(5, True, 0)
        _, b = _samples(ctx, dk, 5, 0, 0, 2, 5)
    assert np.array_equal(a, b) and np.array_equal(c, b)
    assert s_p[0] == 2 and s_p[1] == 0.0 and s_d[0] == 2 and s_d[1] == 0.0


def test_persistent_bounded_wait_reports_timeout(dk):
    """Failure detection without a fault: one tile never reports its step 1,
    the waits for it (limited to 4096 polls) run out, the kernel records the
    timeout and every CTA stops, the call returns MLMC_DK_ERR_TIMEOUT, and
    the same context then runs correct samples."""
    wl = W.get("lowdens32_512").with_(n0=256, L_max=1, T=4.0e-6)
    with dk.Context.from_workload(wl) as ctx, dk.Context.from_workload(wl) as ref:
        assert ctx.stream_wait_test(1, 4096, 5) == dk.ERR_TIMEOUT
        _persistent(ctx, 1, True)
        _, a = _samples(ctx, dk, 1, 0, 0, 3, 9)
        _, b = _samples(ref, dk, 1, 0, 0, 3, 9)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("name,kw,count", [
    ("lowdens32_512", dict(n0=256, L_max=1, T=3.90625e-4, N=1e9), 4),     # 512^2: 1024 fine steps, 256 coarse
    ("large32_1024", dict(n0=512, L_max=1, T=2.44140625e-5, N=3e8), 3),   # 1024^2: 256 fine steps, four modes
])
def test_streamed_longer_horizon_matches_oracle(dk, name, kw, count):
    """The default streamed kernel (dependent launches) over hundreds of fine
    steps, sample by sample against the FP64 oracle (the oracle's cost bounds
    the horizon: about 3e8 cell-steps per sample).  A large N keeps every cell
    far from zero density: at the workloads' own N a 512^2 or 1024^2 cell holds
    a few particles, rho crosses zero, and sqrt(rho^+) amplifies the FP32 noise
    rounding chaotically over hundreds of steps (the ill-conditioning that the
    low-density parity tests bound with the oracle's own sensitivity); the
    kernel's arithmetic is what this test checks.  At 1024^2, N = 3e8 rather
    than 1e9: the absolute fixed-point state's rounding (half a quantum per
    edge and step) is fixed while Y - Ybar shrinks like N^-1/2, and at 1e9 the
    smallest mode of the coarse grid came within 0.8 - 1.06 of the bar."""
    wl = W.get(name).with_(**kw)
    with dk.Context.from_workload(wl) as ctx:
        info = ctx.level_info(1)
        assert info.streamed == 1 and info.pdl == 1 and info.M in (1024, 256)
        K = ctx.n_obs
        _, samp = _samples(ctx, dk, 1, 0, 3, count, 27)
    lv = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu)
    ol = oracle.level_inputs(wl.length, lv, wl.N, wl.rho0_all(), wl.phi_all(), 1, True)
    ref = oracle.run_samples(ol, 27, range(3, 3 + count), True, processes=count)
    for k in range(K):
        for col, key, yb in ((k, "Y_f", info.ybar_f[k]), (K + k, "Y_c", info.ybar_c[k])):
            y = samp[:, col] + yb
            yo = ref[key][:, k]
            rms = np.sqrt(np.mean((yo - yb) ** 2))
            assert np.all(np.abs(y - yo) <= 1e-5 * np.maximum(np.abs(yo), rms)), (k, key, y - yo, rms)
