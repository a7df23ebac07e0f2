"""CPU checks of the C-ABI library: it loads without a GPU, exports every
function include/*.h declares, and its host-only logic (the FFT mean field and
Algorithm 1's planning step) agrees with the FP64 oracle."""
import ctypes
import glob
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2311_08872_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dk():
    libbuild.build()
    from paper_2311_08872_gb300 import mlmc_dk
    return mlmc_dk


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(mlmc_dk_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_function(dk):
    names = _declared_functions()
    assert len(names) >= 15
    L = ctypes.CDLL(dk.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert dk.lib().mlmc_dk_version().startswith(b"mlmc_dk")


@pytest.mark.parametrize("n,mu,M", [(8, 0.1, 30), (32, 0.25, 200), (64, 0.098, 832)])
def test_host_mean_field_matches_oracle_iteration(dk, n, mu, M):
    L = 1.0
    h = L / n
    x = np.arange(n) * h
    x1, x2 = np.meshgrid(x, x, indexing="ij")
    rho0 = 0.02 + 0.98 * np.exp(-((x1 - 0.5) ** 2 + (x2 - 0.4) ** 2) / 0.02) + 0.3 * np.cos(4 * math.pi * x2)
    got = dk.mean_field_host(n, h, mu * h * h, M, rho0)
    ref = oracle.mean_field(n, h, mu * h * h, M, rho0)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_plan_matches_oracle_allocation_and_stopping_test(dk):
    rng = np.random.default_rng(3)
    for trial in range(200):
        L = int(rng.integers(0, 6))
        n = [int(rng.integers(2, 10 ** 6)) for _ in range(L + 1)]
        E = [float(rng.normal(0, 10.0 ** -rng.uniform(1, 5))) for _ in range(L + 1)]
        V = [float(10.0 ** -rng.uniform(1, 8)) for _ in range(L + 1)]
        s1 = [e * m for e, m in zip(E, n)]
        s2 = [(v * (m - 1) + e * e * m) for e, v, m in zip(E, V, n)]
        cost = [float(4.0 ** l * 1e4) for l in range(L + 1)]
        eps = float(10.0 ** -rng.uniform(1, 4))
        targets, conv = dk.plan(n, s1, s2, cost, eps)
        Vh = [max(0.0, (b - a * a / m) / (m - 1)) for a, b, m in zip(s1, s2, n)]
        Eh = [a / m for a, m in zip(s1, n)]
        ref = oracle.mlmc_optimal_samples(Vh, cost, eps)
        for t, r, m in zip(targets, ref, n):
            # ceil of the same real number; allow one unit for rounding order
            assert abs(t - max(r, m)) <= 1 or t == m
        assert conv == oracle.mlmc_converged(Eh, eps)


def test_init_reports_errors_without_crashing(dk):
    one = [np.ones((4, 4))]
    phi = [[np.ones((4, 4))]]
    with pytest.raises(dk.MLMCError) as e:   # mu > 1/2 violates the discrete maximum principle
        dk.Context(1.0, 4, 0, 1.0, 0.6, 100.0, one, phi)
    assert e.value.code == dk.ERR_INVALID
    with pytest.raises(dk.MLMCError) as e:   # n0 not a power of two
        dk.Context(1.0, 6, 0, 1.0, 0.1, 100.0, [np.ones((6, 6))], [[np.ones((6, 6))]])
    assert e.value.code == dk.ERR_INVALID


def test_init_without_gpu_fails_loudly(dk):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    one = [np.ones((4, 4))]
    with pytest.raises(dk.MLMCError) as e:
        dk.Context(1.0, 4, 0, 0.01, 0.1, 100.0, one, [[np.ones((4, 4))]])
    assert e.value.code == dk.ERR_CUDA


def test_theta_scheme_config_checks(dk):
    """Weights of Eq. (FullyDiscreteDK): b0 in [0, 1]; with b1 > b0 the step
    ratio is bounded by 1 / (2 (b1 - b0)); the theta kernel covers grids up to
    128^2 and a bounded number of solve steps."""
    one = [np.ones((4, 4))]
    phi = [[np.ones((4, 4))]]
    cases = [(dict(theta_b0=1.5), 0.1, 4, dk.ERR_INVALID),
             (dict(theta_b0=0.25), 1.2, 4, dk.ERR_INVALID),
             (dict(theta_b0=1.0), 25.0, 4, dk.ERR_UNSUPPORTED),
             (dict(theta_b0=0.5), 3.0, 256, dk.ERR_UNSUPPORTED)]
    for kw, mu, n0, code in cases:
        r = [np.ones((n0, n0))]
        with pytest.raises(dk.MLMCError) as e:
            dk.Context(1.0, n0, 0, 1.0, mu, 100.0, r, [[np.ones((n0, n0))]], **kw)
        assert e.value.code == code, (kw, mu, n0)
    import torch
    if not torch.cuda.is_available():
        # a valid theta configuration passes the checks and fails only for want of a GPU
        with pytest.raises(dk.MLMCError) as e:
            dk.Context(1.0, 4, 0, 1.0, 0.9, 100.0, one, phi, theta_b0=0.25)
        assert e.value.code == dk.ERR_CUDA


@pytest.mark.parametrize("alpha", [0.01, 0.21, 0.85, 2.0])
def test_chebyshev_schedule_solves_the_implicit_system(dk, alpha):
    """The kernel's iteration (u = 0, r = b, d = r/(1+4 alpha); u += d, r -= A d,
    d = c1 d + c2 r) with the host's schedule, run in FP64, against the
    oracle's exact Fourier solve of (I + alpha L) u = b."""
    K, c1, c2 = dk.chebyshev_schedule(alpha)
    assert 1 <= K <= 64
    n = 16
    rng = np.random.default_rng(5)
    b = rng.standard_normal((n, n))
    L = lambda a: 4 * a - np.roll(a, 1, 0) - np.roll(a, -1, 0) - np.roll(a, 1, 1) - np.roll(a, -1, 1)
    u = np.zeros_like(b)
    r = b.copy()
    d = r / (1 + 4 * alpha)
    for k in range(K):
        ad = d + alpha * L(d)
        u += d
        r -= ad
        if k + 1 < K:
            d = float(c1[k]) * d + float(c2[k]) * r
    exact = oracle.helmholtz_solve(n, alpha, b)
    # 2^-27 bound of the polynomial, plus the FP32 rounding of the coefficients
    assert np.linalg.norm(u - exact) <= 1e-6 * np.linalg.norm(exact)
    assert dk.chebyshev_schedule(0.0)[0] == 0


@pytest.mark.parametrize("n", [18, 54, 162])
def test_fourier_restriction_matrix_is_the_oracles(dk, n):
    """P1 S P1^T from the host's matrix equals the oracle's restriction (its own
    DFT sums) to FP32 accuracy, and P1 has orthonormal rows."""
    P1 = dk.fourier_restriction(n).astype(np.float64)
    nc = n // 3
    np.testing.assert_allclose(P1 @ P1.T, np.eye(nc), rtol=0, atol=2e-6)
    S = np.random.default_rng(n).standard_normal((n, n))
    np.testing.assert_allclose(P1 @ S @ P1.T, oracle.fourier_restrict(n, nc, S), rtol=0, atol=2e-5)


def test_plan_with_mesh_ratio_three(dk):
    """Eq. (convergence_criterion) on a ratio-3 hierarchy (Fourier coupling)
    against the oracle's test with the same ratio; the allocation does not
    depend on the ratio."""
    rng = np.random.default_rng(11)
    differs = 0
    for trial in range(300):
        L = int(rng.integers(0, 5))
        n = [int(rng.integers(2, 10 ** 5)) for _ in range(L + 1)]
        E = [float(rng.normal(0, 10.0 ** -rng.uniform(1, 4))) for _ in range(L + 1)]
        V = [float(10.0 ** -rng.uniform(1, 8)) for _ in range(L + 1)]
        s1 = [e * m for e, m in zip(E, n)]
        s2 = [(v * (m - 1) + e * e * m) for e, v, m in zip(E, V, n)]
        cost = [float(9.0 ** l * 1e3) for l in range(L + 1)]
        eps = float(10.0 ** -rng.uniform(1, 4))
        t3, c3 = dk.plan(n, s1, s2, cost, eps, ratio=3.0)
        t2, c2 = dk.plan(n, s1, s2, cost, eps)
        assert t3 == t2
        Eh = [a / m for a, m in zip(s1, n)]
        assert c3 == oracle.mlmc_converged(Eh, eps, ratio=3.0)
        differs += c3 != c2
    assert differs > 0      # the ratio changes some decisions


@pytest.mark.parametrize("n,M", [(6, 8), (18, 72), (54, 648)])
def test_host_mean_field_on_fourier_grids(dk, n, M):
    """The mean field the context uses on the Fourier coupling's grids (not
    powers of two: direct stencil steps) against the oracle's iteration."""
    h = 1.0 / n
    x = np.arange(n) * h
    x1, x2 = np.meshgrid(x, x, indexing="ij")
    rho0 = 1.0 + 0.5 * np.sin(2 * math.pi * x1) * np.sin(2 * math.pi * x2) + 0.1 * np.cos(4 * math.pi * x1)
    tau = 0.09 * h * h
    np.testing.assert_allclose(dk.mean_field_host(n, h, tau, M, rho0), oracle.mean_field(n, h, tau, M, rho0),
                               rtol=0, atol=1e-13)


@pytest.mark.parametrize("b0,mu,M", [(0.5, 0.85, 96), (1.0, 1.7, 48), (0.25, 0.9, 30)])
def test_host_theta_mean_field_matches_oracle(dk, b0, mu, M):
    """The theta-scheme mean field of the context (Fourier symbol) against the
    oracle's iterated exact solves."""
    n = 32
    h = 1.0 / n
    x = np.arange(n) * h
    x1, x2 = np.meshgrid(x, x, indexing="ij")
    rho0 = 0.02 + 0.98 * np.exp(-((x1 - 0.5) ** 2 + (x2 - 0.4) ** 2) / 0.02)
    np.testing.assert_allclose(dk.mean_field_host(n, h, mu * h * h, M, rho0, b0=b0),
                               oracle.mean_field(n, h, mu * h * h, M, rho0, b0=b0), rtol=0, atol=1e-12)


def test_fourier_coupling_config_checks(dk):
    """The Fourier hierarchy's configuration checks run before any GPU call:
    an unknown coupling, grids other than 6^2/18^2/54^2/162^2, and the Fourier
    coupling with the theta-scheme are refused."""
    def ctx(n0, L_max, **kw):
        n = [n0 * 3 ** l for l in range(L_max + 1)]
        return dk.Context(1.0, n0, L_max, 0.02, 0.1, 1e5, [np.ones((m, m)) for m in n],
                          [[np.ones((m, m))] for m in n], **kw)
    cases = [(dict(coupling=2), 6, 1, dk.ERR_INVALID),
             (dict(coupling=1), 12, 1, dk.ERR_UNSUPPORTED),
             (dict(coupling=1), 6, 4, dk.ERR_UNSUPPORTED),
             (dict(coupling=1, theta_b0=0.5), 6, 1, dk.ERR_UNSUPPORTED)]
    for kw, n0, L, code in cases:
        with pytest.raises(dk.MLMCError) as e:
            ctx(n0, L, **kw)
        assert e.value.code == code, (kw, n0, L)
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(dk.MLMCError) as e:
            ctx(6, 2, coupling=1)
        assert e.value.code == dk.ERR_CUDA


def _oracle_round(wl):
    """Round sampler from the FP64 oracle: sums in the device layout."""
    levels = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu, wl.M0)
    rho0, phi = wl.rho0_all(), wl.phi_all()
    ybar = [oracle.inner_h(oracle.mean_field(l.n, l.h, l.tau, l.M, rho0[l.level]), phi[l.level][0], l.h)
            for l in levels]

    def dP(l, first, count):
        ol = oracle.level_inputs(wl.length, levels, wl.N, rho0, phi, l, l > 0)
        r = oracle.run_samples(ol, wl.seed, range(first, first + count), l > 0)
        pf = oracle.observable_P(wl.N, r["Y_f"][:, :1], [ybar[l]])[:, 0]
        pc = oracle.observable_P(wl.N, r["Y_c"][:, :1], [ybar[l - 1]])[:, 0] if l else np.zeros(count)
        return pf, pc

    cost = [levels[l].n ** 2 * levels[l].M + (levels[l - 1].n ** 2 * levels[l - 1].M if l else 0)
            for l in range(len(levels))]
    return dP, cost


def test_algorithm1_in_the_library_matches_the_oracles_statement(dk):
    """mlmc_dk_algorithm1 (the library's Algorithm 1, Section 7.1) with oracle
    samples, against Algorithm 1 written out with the oracle's Eq. (opt_M_ell),
    Eq. (convergence_criterion) and Eq. (MLMCEstimator) on the same samples:
    the same levels, sample counts and estimate."""
    from paper_2311_08872_gb300 import workloads as W
    wl = W.get("mlmc16_256").with_(n0=8, L_max=3, T=0.005, N=1e5)
    dP, cost = _oracle_round(wl)
    cache = {}

    def samples(l, first, count):
        pf, pc = dP(l, first, count)
        for i in range(count):
            cache[(l, first + i)] = (pf[i], pc[i])
        return pf, pc

    def run_round(L, first, count):
        out = np.zeros((wl.L_max + 1, 14))
        for l in range(wl.L_max + 1):
            if count[l] > 0:
                pf, pc = samples(l, first[l], count[l])
                d = pf - pc
                out[l, :10] = [count[l], 0.0, d.sum(), (d ** 2).sum(), (d ** 3).sum(), (d ** 4).sum(),
                               pf.sum(), (pf ** 2).sum(), pc.sum(), (pc ** 2).sum()]
        return out

    r = dk.algorithm1(run_round, None, wl.L_max, 1, cost, 0.03, pilot=64, L_start=2)
    # the same algorithm from the oracle's formulas, on the cached samples
    L, target, n = 2, [64, 64, 64, 0], [0, 0, 0, 0]
    eps_abs = None
    while True:
        for l in range(L + 1):
            n[l] = max(n[l], target[l])
        d = [np.array([cache[(l, i)][0] - cache[(l, i)][1] for i in range(n[l])]) for l in range(L + 1)]
        E = [x.mean() for x in d]
        V = [x.var(ddof=1) for x in d]
        if eps_abs is None:
            eps_abs = 0.03 * abs(sum(E))
        opt = oracle.mlmc_optimal_samples(V, cost[:L + 1], eps_abs)
        more = False
        for l in range(L + 1):
            target[l] = max(target[l], opt[l], n[l])
            if target[l] - n[l] > 0.01 * n[l]:
                more = True
        if more:
            if any((l, target[l] - 1) not in cache for l in range(L + 1)):
                break        # the library stopped earlier than this statement would: fails below
            continue
        if oracle.mlmc_converged(E, eps_abs) or L == wl.L_max:
            break
        L += 1
        target[L] = 64
    assert r.L == L
    assert [r.M[l] for l in range(L + 1)] == n[:L + 1]
    est = oracle.mlmc_estimator([x.sum() for x in d], [x.size for x in d])
    assert r.estimate == pytest.approx(est, rel=1e-12)
    assert r.eps_abs == pytest.approx(eps_abs, rel=1e-12)
