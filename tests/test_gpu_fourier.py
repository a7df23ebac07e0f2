"""GPU parity of the Fourier-coupled kernel (Section 3.1: h ratio 3, tau
ratio 9, the coarse noise carrying every resolved Fourier mode of the fine
noise) against the FP64 oracle, through the C-ABI; and the coupling's
properties on the GPU: the coarse member's law equals a stand-alone coarse
path's (Remark distribution_W_ell), Var[P_l - P_{l-1}] falls faster than the
NN coupling's rate (Proposition PropBoundVarLevels: beta = 4 against 2), and
Algorithm 1 runs on the ratio-3 hierarchy.
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


def _levels(wl):
    return oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu, wl.M0, ratio=3)


def _ybar(wl, levels, l):
    lv = levels[l]
    return np.array([oracle.inner_h(oracle.mean_field(lv.n, lv.h, lv.tau, lv.M, wl.rho0(l)), p, lv.h)
                     for p in wl.phi(l)])


@pytest.mark.parametrize("level,tag,count", [(0, 0, 32), (1, 0, 24), (2, 0, 8), (2, 1, 6)])
def test_fourier_kernel_matches_oracle(dk, level, tag, count):
    wl = W.get("fourier6_54")
    seed, first = 41 + level, 3
    levels = _levels(wl)
    with dk.Context.from_workload(wl) as ctx:
        info = ctx.level_info(level)
        assert info.coupling == 1 and info.n == levels[level].n and info.M == levels[level].M
        sums, samp = _gpu(ctx, dk, level, tag, first, count, seed)
    coupled = tag == 0 and level > 0
    ol = oracle.level_inputs(wl.length, levels, wl.N, wl.rho0_all(), wl.phi_all(), level, coupled, coupling=1)
    r = oracle.run_samples(ol, seed, range(first, first + count), coupled, stream=tag)
    ybf = _ybar(wl, levels, level)
    np.testing.assert_allclose(np.array(info.ybar_f[:1]), ybf, rtol=1e-9, atol=1e-12)
    worst = 0.0
    pairs = [(samp[:, 0] + ybf[0], r["Y_f"][:, 0], ybf[0])]
    if coupled:
        ybc = _ybar(wl, levels, level - 1)
        np.testing.assert_allclose(np.array(info.ybar_c[:1]), ybc, rtol=1e-9, atol=1e-12)
        pairs.append((samp[:, 1] + ybc[0], r["Y_c"][:, 0], ybc[0]))
    for y, yo, yb in pairs:
        scale = np.sqrt(np.mean((yo - yb) ** 2))
        w = float(np.max(np.abs(y - yo) / (TOL * np.maximum(np.abs(yo), scale))))
        assert w <= 1.0, f"level {level} tag {tag}: worst error / bound = {w:.3g}"
        worst = max(worst, w)
    assert int(sums[0]) == count and sums[1] == 0.0
    print(f"fourier6_54 level {level} tag {tag}: worst/bound {worst:.3g}")


def test_coarse_member_law_and_variance_decay(dk):
    """E[P_c] of level-l pairs equals E[P_f] of stand-alone level-(l-1) paths,
    and V_l decays like h^beta with beta well above the NN coupling's 2 at
    high density (the paper predicts 4 for the Fourier coupling)."""
    wl = W.get("fourier6_54").with_(N=1e9)
    with dk.Context.from_workload(wl) as ctx:
        s1 = ctx.run_level(1, 200000, 7)[0]
        s2 = ctx.run_level(2, 20000, 8)[0]
        a0 = ctx.run_level(0, 200000, 9, mc=True)[0]
        a1 = ctx.run_level(1, 20000, 10, mc=True)[0]
    var = lambda s: (s.dp2 - s.dp1 ** 2 / s.n) / (s.n - 1)
    for pair, alone in ((s1, a0), (s2, a1)):
        mc, ma = pair.pc1 / pair.n, alone.pf1 / alone.n
        vc = (pair.pc2 - pair.pc1 ** 2 / pair.n) / (pair.n - 1)
        va = (alone.pf2 - alone.pf1 ** 2 / alone.n) / (alone.n - 1)
        assert abs(mc - ma) < 4.0 * math.sqrt(vc / pair.n + va / alone.n), (mc, ma)
    v1, v2 = var(s1), var(s2)
    beta = math.log(v1 / v2) / math.log(3.0)
    print(f"Fourier coupling at N = 1e9: V_1 = {v1:.3e}, V_2 = {v2:.3e}, beta = {beta:.2f}")
    assert beta > 2.5


def test_algorithm1_on_fourier_levels(dk):
    wl = W.get("fourier6_54")
    with dk.Context.from_workload(wl) as ctx:
        r = ctx.estimate(2e-2, True, 5)
        assert r.L >= 1 and all(r.M[l] > 0 for l in range(r.L + 1))
        assert math.isfinite(r.estimate) and r.estimate > 0


def test_empty_batch_gives_zero_sums(dk):
    wl = W.get("fourier6_54")
    with dk.Context.from_workload(wl) as ctx:
        sums, _ = _gpu(ctx, dk, 2, 0, 0, 0, 1)
    assert not sums.any()


def test_four_observables_with_products(dk):
    four = W.get("large32_1024").observables
    wl = W.get("fourier6_54").with_(name="fourier6_54_four", observables=four, products=True)
    level, count, seed, first = 1, 12, 73, 0
    levels = _levels(wl)
    with dk.Context.from_workload(wl) as ctx:
        assert ctx.n_quant == 10
        sums, samp = _gpu(ctx, dk, level, 0, first, count, seed)
    ol = oracle.level_inputs(wl.length, levels, wl.N, wl.rho0_all(), wl.phi_all(), level, True, coupling=1)
    r = oracle.run_samples(ol, seed, range(first, first + count), True)
    for cols, key, l in ((slice(0, 4), "Y_f", level), (slice(4, 8), "Y_c", level - 1)):
        yb = _ybar(wl, levels, l)
        yo = r[key]
        scale = np.sqrt(np.mean((yo - yb[None, :]) ** 2, axis=0))
        err = np.abs(samp[:, cols] + yb[None, :] - yo) / (TOL * np.maximum(np.abs(yo), scale[None, :]))
        assert float(err.max()) <= 1.0, (key, float(err.max()))
    assert int(sums[0]) == count and sums[1] == 0.0


# ---------------------------------------------------------------- 162^2 on clusters
def _short162():
    """The four-level hierarchy over one level-0 step (T = tau_0 = 0.0025,
    tau/h^2 = 0.09): 729 fine and 81 coarse steps on the 162^2 level, so that
    the oracle's samples take seconds."""
    return W.get("fourier6_162").with_(name="fourier6_162_short", T=0.0025, M0=1)


def _worst(wl, levels, level, coupled, samp, r):
    ybf = _ybar(wl, levels, level)
    pairs = [(samp[:, 0] + ybf[0], r["Y_f"][:, 0], ybf[0])]
    if coupled:
        ybc = _ybar(wl, levels, level - 1)
        pairs.append((samp[:, 1] + ybc[0], r["Y_c"][:, 0], ybc[0]))
    worst = 0.0
    for y, yo, yb in pairs:
        scale = np.sqrt(np.mean((yo - yb) ** 2))
        worst = max(worst, float(np.max(np.abs(y - yo) / (TOL * np.maximum(np.abs(yo), scale)))))
    return worst


@pytest.mark.parametrize("tag,count", [(0, 6), (1, 4)])
def test_fourier_cluster_level_162_matches_oracle(dk, tag, count):
    """The 162^2 level (coupled with 54^2) runs on the cluster kernel: 6 CTAs
    per sample, the neighbouring rows and the partial restrictions of the
    coarse noise through distributed shared memory.  Per-sample parity with the
    oracle for the coupled pair (tag 0) and the fine path alone (tag 1)."""
    wl = _short162()
    level, seed, first = 3, 51 + tag, 5
    levels = _levels(wl)
    assert levels[level].n == 162 and levels[level].M == 729
    with dk.Context.from_workload(wl) as ctx:
        info = ctx.level_info(level)
        assert info.coupling == 1 and info.n == 162 and info.M == 729 and info.cluster == 6
        sums, samp = _gpu(ctx, dk, level, tag, first, count, seed)
    coupled = tag == 0
    ol = oracle.level_inputs(wl.length, levels, wl.N, wl.rho0_all(), wl.phi_all(), level, coupled, coupling=1)
    r = oracle.run_samples(ol, seed, range(first, first + count), coupled, stream=tag, processes=count)
    worst = _worst(wl, levels, level, coupled, samp, r)
    print(f"fourier6_162 level 3 tag {tag}: worst/bound {worst:.3g}")
    assert worst <= 1.0
    # the integer flux form conserves the (quantised) initial mass exactly
    for col, key, l in ((2, "mass_f", level), (3, "mass_c", level - 1))[:2 if coupled else 1]:
        m0 = oracle.inner_h(wl.rho0(l), np.ones_like(wl.rho0(l)), levels[l].h)
        np.testing.assert_allclose(samp[:, col], m0, rtol=1e-7)
        assert np.ptp(samp[:, col]) == 0.0
        np.testing.assert_allclose(r[key], m0, rtol=1e-12)
    assert int(sums[0]) == count and sums[1] == 0.0


def test_fourier_cluster_level_many_samples_and_batch(dk):
    """More samples than resident clusters (several passes of the persistent
    cluster grid, a ragged last pass): device sums equal the per-sample
    outputs' sums, and the multi-level batch gives the same sums as per-level
    launches with the 162^2 level in it."""
    import torch
    wl = _short162()
    st = torch.cuda.current_stream().cuda_stream
    with dk.Context.from_workload(wl) as ctx:
        info = ctx.level_info(3)
        count = 2 * (info.in_flight or 24) + 5
        sums, samp = _gpu(ctx, dk, 3, 0, 0, count, 14)
        assert int(sums[0]) == count and sums[1] == 0.0
        dp = wl.N * (samp[:, 0] ** 2 - samp[:, 1] ** 2)
        np.testing.assert_allclose(sums[2], dp.sum(), rtol=1e-9)
        S = dk.sums_len(ctx.n_quant)
        counts = [400, 100, 30, 20]
        batch = torch.zeros(4, S, dtype=torch.float64, device="cuda")
        ctx.run_batch_dev(counts, 3, 15, batch.data_ptr(), st)
        torch.cuda.synchronize()
        for l, m in enumerate(counts):
            ref = torch.zeros(S, dtype=torch.float64, device="cuda")
            ctx.run_level_dev(l, 0, 3, m, 15, ref.data_ptr(), 0, st)
            torch.cuda.synchronize()
            np.testing.assert_allclose(batch[l].cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=0)


def test_fourier_162_coarse_member_law_and_variance_decay(dk):
    """Full horizon (5832 fine steps at 162^2): E[P_c] of level-3 pairs equals
    E[P_f] of stand-alone 54^2 paths (Remark distribution_W_ell), the mass
    stays exact, and V_3 / V_2 falls like 3^-beta with beta well above the NN
    coupling's 2 (the paper predicts 4)."""
    wl = W.get("fourier6_162").with_(N=1e9)
    with dk.Context.from_workload(wl) as ctx:
        s3 = ctx.run_level(3, 1500, 21)[0]
        s2 = ctx.run_level(2, 20000, 22)[0]
        a2 = ctx.run_level(2, 20000, 23, mc=True)[0]
    var = lambda s: (s.dp2 - s.dp1 ** 2 / s.n) / (s.n - 1)
    mc, ma = s3.pc1 / s3.n, a2.pf1 / a2.n
    vc = (s3.pc2 - s3.pc1 ** 2 / s3.n) / (s3.n - 1)
    va = (a2.pf2 - a2.pf1 ** 2 / a2.n) / (a2.n - 1)
    assert abs(mc - ma) < 4.0 * math.sqrt(vc / s3.n + va / a2.n), (mc, ma)
    assert s3.max_mass_err < 1e-12
    v2, v3 = var(s2), var(s3)
    beta = math.log(v2 / v3) / math.log(3.0)
    print(f"Fourier coupling at N = 1e9: V_2 = {v2:.3e}, V_3 = {v3:.3e}, beta = {beta:.2f}")
    assert beta > 2.5


def test_algorithm1_reaches_162_and_matches_closed_form(dk):
    """Algorithm 1 on the four-level hierarchy (6^2 .. 162^2) at N = 1e9 and
    eps = 1e-3 relative: the stopping test of Eq. (convergence_criterion) with
    ratio 3 needs the 162^2 level, the estimator variance meets eps^2 / 2, and
    the estimate is within 4 standard deviations of the closed form of E[P_3]
    (the telescoping sum is unbiased for the finest level's expectation, and
    at N = 1e9 the density stays positive, so the closed form is exact)."""
    wl = W.get("fourier6_162").with_(N=1e9)
    with dk.Context.from_workload(wl) as ctx:
        r = ctx.estimate(1e-3, relative=True, seed=wl.seed)
        info = ctx.level_info(r.L)
    print("estimate", r.estimate, "L", r.L, "M", [r.M[l] for l in range(r.L + 1)], "wall", r.wall_s)
    assert r.L == 3 and r.converged == 1 and info.n == 162
    assert r.variance <= r.eps_abs ** 2 / 2 * 1.05
    cf = oracle.closed_form_EP_cos1(1.0, info.n, info.tau, info.M)
    assert abs(r.estimate - cf) < 4 * math.sqrt(r.variance), (r.estimate, cf, math.sqrt(r.variance))


# ---------------------------------------------------------------- fluctuation state
@pytest.mark.parametrize("level,tag,count", [(1, 0, 12), (2, 0, 8), (2, 1, 6)])
def test_paper_setting_fourier_main_particle_number(dk, level, tag, count):
    """The paper's regular setting (Section 7.2) with the Fourier coupling at
    its main particle number N = 2e9: the state is held as its fluctuation
    about the noise-free path (chosen automatically), meets the unrelaxed
    per-sample bar, and the reported masses are the mean field's."""
    wl = W.get("paper_reg_fourier")
    levels = _levels(wl)
    seed, first = wl.seed, 3
    with dk.Context.from_workload(wl) as ctx:
        assert all(ctx.level_info(l).fluct == 1 for l in range(wl.L_max + 1))
        sums, samp = _gpu(ctx, dk, level, tag, first, count, seed)
    coupled = tag == 0
    ol = oracle.level_inputs(wl.length, levels, wl.N, wl.rho0_all(), wl.phi_all(), level, coupled, coupling=1)
    r = oracle.run_samples(ol, seed, range(first, first + count), coupled, stream=tag, processes=4)
    worst = _worst(wl, levels, level, coupled, samp, r)
    print(f"paper_reg_fourier N = 2e9 level {level} tag {tag}: worst/bound {worst:.3g}")
    assert worst <= 1.0
    np.testing.assert_allclose(samp[:, 2], r["mass_f"], rtol=1e-12)
    if coupled:
        np.testing.assert_allclose(samp[:, 3], r["mass_c"], rtol=1e-12)
    assert int(sums[0]) == count and sums[1] == 0.0


def test_fluctuation_state_on_request_at_low_particle_number(dk):
    """The fluctuation state asked for explicitly where the automatic choice is
    the absolute one (N = 1e5): the same scheme, so the same per-sample bar
    against the oracle; the 162^2 level has no such build and is refused."""
    wl = W.get("fourier6_54")
    levels = _levels(wl)
    level, seed, first, count = 2, 61, 0, 8
    with dk.Context.from_workload(wl) as ctx:
        assert ctx.level_info(level).fluct == 0
    with dk.Context.from_workload(wl, state_repr=2) as ctx:
        assert ctx.level_info(level).fluct == 1
        sums, samp = _gpu(ctx, dk, level, 0, first, count, seed)
    ol = oracle.level_inputs(wl.length, levels, wl.N, wl.rho0_all(), wl.phi_all(), level, True, coupling=1)
    r = oracle.run_samples(ol, seed, range(first, first + count), True, processes=4)
    worst = _worst(wl, levels, level, True, samp, r)
    print(f"fourier6_54 fluctuation state at N = 1e5: worst/bound {worst:.3g}")
    assert worst <= 1.0 and sums[1] == 0.0
    with pytest.raises(dk.MLMCError) as e:
        dk.Context.from_workload(W.get("fourier6_162"), state_repr=2)
    assert e.value.code == dk.ERR_UNSUPPORTED
