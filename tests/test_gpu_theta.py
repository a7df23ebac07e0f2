"""GPU parity of the theta-scheme kernel (Eq. FullyDiscreteDK with b0 > 0)
against the FP64 oracle, through the C-ABI.

* b0 = 0 on the theta-scheme kernel is the explicit step with the same
  integer arithmetic: identical states to the streamed kernels (both project
  on FP64 test functions, so Y agrees to FP64 summation order) and the
  register kernels' observables within their FP32 partial sums.
* Crank--Nicolson (b0 = 1/2, tau/h^2 = 0.85) and implicit Euler (b0 = 1,
  tau/h^2 = 1.7), beyond the explicit limit 1/2: per-sample Y of the fine and
  coupled coarse paths within 1e-5 of the fluctuation scale of the oracle's
  exact Fourier solve, exact mass, the discrete mean field of the theta
  symbol.
* E[P] on the GPU against the martingale closed form with the solve's
  factor on the noise, and E[Y] = Ybar.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_08872_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def dk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2311_08872_gb300 import build as libbuild
    libbuild.build()
    from paper_2311_08872_gb300 import mlmc_dk
    return mlmc_dk


def _gpu(ctx, dk, level, tag, first, count, seed):
    import torch
    sums = torch.zeros(dk.sums_len(ctx.n_quant), dtype=torch.float64, device="cuda")
    samp = torch.zeros(max(count, 1), dk.sample_stride(ctx.n_obs), dtype=torch.float64, device="cuda")
    ctx.run_level_dev(level, tag, first, count, seed, sums.data_ptr(), samp.data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return sums.cpu().numpy(), samp.cpu().numpy()[:count]


def _oracle(wl, level, tag, first, count, seed):
    levels = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu, wl.M0)
    coupled = tag == 0 and level > 0
    ol = oracle.level_inputs(wl.length, levels, wl.N, wl.rho0_all(), wl.phi_all(), level, coupled, b0=wl.b0)
    r = oracle.run_samples(ol, seed, range(first, first + count), coupled, stream=tag)
    ybar = lambda l: np.array([oracle.inner_h(oracle.mean_field(levels[l].n, levels[l].h, levels[l].tau, levels[l].M,
                                                                wl.rho0(l), b0=wl.b0), p, levels[l].h)
                               for p in wl.phi(l)])
    return r, ybar(level), (ybar(level - 1) if coupled else None)


def _parity(y_gpu, y_or, ybar, what):
    scale = np.sqrt(np.mean((y_or - ybar[None, :]) ** 2, axis=0))
    bound = TOL * np.maximum(np.abs(y_or), scale[None, :])
    worst = float(np.max(np.abs(y_gpu - y_or) / bound))
    assert worst <= 1.0, f"{what}: worst error / bound = {worst:.3g}"
    return worst


@pytest.mark.parametrize("name,level,tag,count", [
    ("theta16_64", 0, 0, 24), ("theta16_64", 1, 0, 16), ("theta16_64", 2, 0, 8), ("theta16_64", 2, 1, 8),
    ("implicit16_64", 1, 0, 16), ("implicit16_64", 2, 0, 8)])
def test_theta_kernel_matches_oracle(dk, name, level, tag, count):
    wl = W.get(name)
    seed, first = 31 + level, 5
    with dk.Context.from_workload(wl) as ctx:
        info = ctx.level_info(level)
        assert info.theta == 1 and info.theta_b0 == wl.b0 and info.cheb_steps > 0
        sums, samp = _gpu(ctx, dk, level, tag, first, count, seed)
    r, ybf, ybc = _oracle(wl, level, tag, first, count, seed)
    K = 1
    np.testing.assert_allclose(np.array(info.ybar_f[:K]), ybf, rtol=1e-9, atol=1e-12)
    w = _parity(samp[:, :K] + ybf[None, :], r["Y_f"], ybf, f"{name} level {level} fine")
    if ybc is not None:
        np.testing.assert_allclose(np.array(info.ybar_c[:K]), ybc, rtol=1e-9, atol=1e-12)
        w = max(w, _parity(samp[:, K:2 * K] + ybc[None, :], r["Y_c"], ybc, f"{name} level {level} coarse"))
    assert int(sums[0]) == count
    assert sums[1] == 0.0                    # integer face fluxes: mass exact
    m0 = oracle.inner_h(wl.rho0(level), np.ones_like(wl.rho0(level)), info.h)
    np.testing.assert_allclose(samp[:, 2 * K], m0, rtol=1e-7)
    print(f"{name} level {level} tag {tag}: worst/bound {w:.3g}, Chebyshev steps {info.cheb_steps}")


@pytest.mark.parametrize("name,tag", [("theta16_64", 0), ("theta16_64", 1), ("implicit16_64", 0)])
def test_theta_cluster_level_128_matches_oracle(dk, name, tag):
    """The 128^2 level (coupled with 64^2) runs on the cluster kernel: 4 CTAs
    per sample, each a band of 16 block rows (two blocks per thread),
    neighbour rows through distributed shared memory and cluster barriers.  Full horizon (384 fine
    steps), sample by sample against the oracle's exact Fourier solves."""
    wl = W.get(name).with_(L_max=3)
    level, count, seed, first = 3, 4, 41, 2
    with dk.Context.from_workload(wl) as ctx:
        info = ctx.level_info(level)
        assert info.n == 128 and info.theta == 1 and info.cluster == 4 and info.cheb_steps > 0
        sums, samp = _gpu(ctx, dk, level, tag, first, count, seed)
    levels = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu, wl.M0)
    coupled = tag == 0
    ol = oracle.level_inputs(wl.length, levels, wl.N, wl.rho0_all(), wl.phi_all(), level, coupled, b0=wl.b0)
    r = oracle.run_samples(ol, seed, range(first, first + count), coupled, stream=tag, processes=4)
    K = 1
    ybf = np.array(info.ybar_f[:K])
    w = _parity(samp[:, :K] + ybf[None, :], r["Y_f"], ybf, f"{name} level 3 fine")
    if coupled:
        ybc = np.array(info.ybar_c[:K])
        w = max(w, _parity(samp[:, K:2 * K] + ybc[None, :], r["Y_c"], ybc, f"{name} level 3 coarse"))
    assert int(sums[0]) == count and sums[1] == 0.0
    print(f"{name} 128^2 tag {tag}: worst/bound {w:.3g}, Chebyshev steps {info.cheb_steps}")


def test_theta_cluster_level_many_samples_and_batch(dk):
    """More samples than resident clusters (several passes of the persistent
    cluster grid, a ragged last pass): device sums equal the per-sample
    outputs' sums, and the multi-level batch gives the same sums as per-level
    launches with the 128^2 level in it."""
    import torch
    wl = W.get("theta16_64").with_(L_max=3, T=0.0025)
    st = torch.cuda.current_stream().cuda_stream
    with dk.Context.from_workload(wl) as ctx:
        info = ctx.level_info(3)
        count = 2 * (info.in_flight or 19) + 3
        sums, samp = _gpu(ctx, dk, 3, 0, 0, count, 12)
        assert int(sums[0]) == count
        dp = wl.N * (samp[:, 0] ** 2 - samp[:, 1] ** 2)
        np.testing.assert_allclose(sums[2], dp.sum(), rtol=1e-9)
        S = dk.sums_len(ctx.n_quant)
        counts = [400, 100, 30, 25]
        batch = torch.zeros(4, S, dtype=torch.float64, device="cuda")
        ctx.run_batch_dev(counts, 3, 13, batch.data_ptr(), st)
        torch.cuda.synchronize()
        for l, m in enumerate(counts):
            ref = torch.zeros(S, dtype=torch.float64, device="cuda")
            ctx.run_level_dev(l, 0, 3, m, 13, ref.data_ptr(), 0, st)
            torch.cuda.synchronize()
            np.testing.assert_allclose(batch[l].cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=0)


def test_b0_zero_theta_kernel_is_the_explicit_step(dk):
    """The theta kernel with b0 = 0 against the streamed kernels (64^2, the same
    integer arithmetic and FP64 projections) and the register kernels (16^2,
    32^2: FP32 partial projections)."""
    wl = W.get("mlmc16_256").with_(L_max=2)
    seed, first = 77, 3
    with dk.Context.from_workload(wl, theta_kernel=True) as th, \
            dk.Context.from_workload(wl, stream_from_n=64) as ex:
        assert th.level_info(2).theta == 1 and th.level_info(2).cheb_steps == 0
        assert ex.level_info(2).streamed == 1 and ex.level_info(1).streamed == 0
        for level, count in ((0, 40), (1, 24), (2, 12)):
            st, sa = _gpu(th, dk, level, 0, first, count, seed)
            se, sb = _gpu(ex, dk, level, 0, first, count, seed)
            assert st[1] == 0.0 and se[1] == 0.0
            np.testing.assert_allclose(sa[:, 2:], sb[:, 2:], rtol=1e-14)   # masses: the same integer sums
            tol = 1e-12 if level == 2 else TOL
            for col in range(2 if level > 0 else 1):
                scale = np.sqrt(np.mean(sb[:, col] ** 2))
                err = np.max(np.abs(sa[:, col] - sb[:, col])) / scale
                assert err <= tol, (level, col, err)


@pytest.mark.parametrize("name", ["theta16_64", "implicit16_64"])
def test_theta_mean_and_second_moment_closed_forms(dk, name):
    """High density (rho stays positive): E[Y_f] = Ybar and E[P_f] equals the
    martingale closed form with the factor 1 / (1 + b0 lam)^2 on the noise."""
    wl = W.get(name).with_(N=1e8)
    n_s = 20000
    with dk.Context.from_workload(wl) as ctx:
        info = ctx.level_info(2)
        s = ctx.run_level(2, n_s, 123, mc=True)[0]
    mean_y = s.yf1 / s.n
    se_y = math.sqrt(max(s.yf2 / s.n - mean_y ** 2, 0.0) / s.n)
    assert abs(mean_y) < 4.0 * se_y
    mean_p = s.pf1 / s.n
    se_p = math.sqrt(max(s.pf2 / s.n - mean_p ** 2, 0.0) / s.n)
    expect = oracle.closed_form_EP_cos1(1.0, info.n, info.tau, info.M, b0=wl.b0)
    assert abs(mean_p - expect) < 4.0 * se_p, (mean_p, expect, se_p)
    assert se_p / expect < 0.03


def test_algorithm1_runs_on_theta_levels(dk):
    wl = W.get("theta16_64")
    with dk.Context.from_workload(wl) as ctx:
        r = ctx.estimate(2e-2, True, 9)
        assert r.L == 2 and all(r.M[l] > 0 for l in range(3))
        assert math.isfinite(r.estimate) and r.estimate > 0
        info = ctx.level_info(2)
        cf = oracle.closed_form_EP_cos1(1.0, info.n, info.tau, info.M, b0=wl.b0)
        assert abs(r.estimate - cf) < 0.1 * cf


@pytest.mark.parametrize("level,count", [(0, 37), (1, 29), (2, 13)])
def test_small_grids_and_ragged_counts(dk, level, count):
    """Grids 4^2, 8^2, 16^2 (several samples per CTA, sub-warp reductions) with
    sample counts that leave the last CTA partly idle."""
    wl = W.get("theta16_64").with_(name="theta4_16", n0=4, L_max=2)
    seed, first = 61 + level, 2
    with dk.Context.from_workload(wl) as ctx:
        info = ctx.level_info(level)
        assert info.theta == 1 and info.n == 4 << level
        sums, samp = _gpu(ctx, dk, level, 0, first, count, seed)
    r, ybf, ybc = _oracle(wl, level, 0, first, count, seed)
    _parity(samp[:, :1] + ybf[None, :], r["Y_f"], ybf, f"theta 4..16 level {level} fine")
    if ybc is not None:
        _parity(samp[:, 1:2] + ybc[None, :], r["Y_c"], ybc, f"theta 4..16 level {level} coarse")
    assert int(sums[0]) == count and sums[1] == 0.0


def test_empty_batch_gives_zero_sums(dk):
    wl = W.get("theta16_64")
    with dk.Context.from_workload(wl) as ctx:
        sums, _ = _gpu(ctx, dk, 2, 0, 0, 0, 1)
    assert not sums.any()


def test_four_observables_with_products(dk):
    """Four test functions and all their products on the theta kernel: every
    observable per sample against the oracle, ten quantities summed."""
    four = W.get("large32_1024").observables
    wl = W.get("theta16_64").with_(name="theta16_64_four", observables=four, products=True)
    level, count, seed, first = 1, 12, 71, 0
    with dk.Context.from_workload(wl) as ctx:
        assert ctx.n_quant == 10
        sums, samp = _gpu(ctx, dk, level, 0, first, count, seed)
    r, ybf, ybc = _oracle(wl, level, 0, first, count, seed)
    _parity(samp[:, 0:4] + ybf[None, :], r["Y_f"], ybf, "theta four observables fine")
    _parity(samp[:, 4:8] + ybc[None, :], r["Y_c"], ybc, "theta four observables coarse")
    assert int(sums[0]) == count and sums[1] == 0.0
