"""Statistical pins for the oracle (k-standard-error checks on seeded runs).

* E[Y_l] equals the discrete mean-field value exactly, at any particle
  density (the scheme is linear in rho and the noise has zero conditional
  mean; Lemma lem_Discrete_Martingale).
* E[P_l] equals the martingale-lemma closed form when rho stays positive.
* The coarse member of an NN-coupled pair has the law of a stand-alone
  coarser path (Remark distribution_W_ell, stated for the NN coupling in
  Section 3.2), which makes the telescoping sum unbiased.
* Var[P_l - P_{l-1}] decays with h_l in the high-density regime
  (Proposition PropBoundVarLevels, beta = 2 for NN coupling).
"""
import math

import numpy as np
import pytest

import oracle

K_SE = 3.5


def _grid(n, L=1.0):
    x = np.arange(n) * (L / n)
    return np.meshgrid(x, x, indexing="ij")


def _sinsin(n):
    x1, x2 = _grid(n)
    return 1.0 + 0.5 * np.sin(2 * math.pi * x1) * np.sin(2 * math.pi * x2)


def _cos1(n):
    x1, _ = _grid(n)
    return np.cos(2 * math.pi * x1)


def _gauss(n):
    x1, x2 = _grid(n)
    out = np.full_like(x1, 0.02)
    for s1 in (-1, 0, 1):
        for s2 in (-1, 0, 1):
            out += 0.98 * np.exp(-((x1 - 0.5 + s1) ** 2 + (x2 - 0.5 + s2) ** 2) / 0.02)
    return out


def _inputs(levels, N, rho0, phi, level, coupled):
    r = [rho0(lv.n) for lv in levels]
    p = [[phi(lv.n)] for lv in levels]
    return oracle.level_inputs(1.0, levels, N, r, p, level, coupled)


@pytest.mark.parametrize("N,rho0", [(1e4, _sinsin), (30.0, _gauss)])
def test_mean_of_Y_is_discrete_mean_field(N, rho0):
    levels = oracle.level_table(1.0, 8, 1, 0.02, 0.1)
    ol = _inputs(levels, N, rho0, _cos1, 1, coupled=True)
    r = oracle.run_samples(ol, seed=123, ids=range(1500), coupled=True)
    for key, lv in (("Y_f", levels[1]), ("Y_c", levels[0])):
        Ybar = oracle.inner_h(oracle.mean_field(lv.n, lv.h, lv.tau, lv.M, rho0(lv.n)), _cos1(lv.n), lv.h)
        y = r[key][:, 0]
        se = y.std(ddof=1) / math.sqrt(y.size)
        assert abs(y.mean() - Ybar) < K_SE * se


def test_mean_of_P_matches_martingale_closed_form():
    N = 1e8   # N h^2 ~ 4e5 particles per cell: rho stays positive
    lv = oracle.level_table(1.0, 16, 0, 0.02, 0.1)[0]
    ol = oracle.OracleLevel(lv, N, _sinsin(16), [_cos1(16)])
    r = oracle.run_samples(ol, seed=7, ids=range(2500), coupled=False, stream=1)
    Ybar = oracle.inner_h(oracle.mean_field(16, lv.h, lv.tau, lv.M, _sinsin(16)), _cos1(16), lv.h)
    P = oracle.observable_P(N, r["Y_f"], [Ybar])[:, 0]
    se = P.std(ddof=1) / math.sqrt(P.size)
    expect = oracle.closed_form_EP_cos1(1.0, 16, lv.tau, lv.M)
    assert abs(P.mean() - expect) < K_SE * se
    assert se / expect < 0.05


def test_coarse_path_has_law_of_standalone_coarse_path():
    N = 2e3
    levels = oracle.level_table(1.0, 8, 1, 0.02, 0.1)
    pair = _inputs(levels, N, _sinsin, _cos1, 1, coupled=True)
    alone = _inputs(levels, N, _sinsin, _cos1, 0, coupled=False)
    rp = oracle.run_samples(pair, seed=5, ids=range(2000), coupled=True)
    ra = oracle.run_samples(alone, seed=5, ids=range(2000), coupled=False, stream=1)
    lv0 = levels[0]
    Ybar0 = oracle.inner_h(oracle.mean_field(8, lv0.h, lv0.tau, lv0.M, _sinsin(8)), _cos1(8), lv0.h)
    Pc = oracle.observable_P(N, rp["Y_c"], [Ybar0])[:, 0]
    Pa = oracle.observable_P(N, ra["Y_f"], [Ybar0])[:, 0]
    se = math.sqrt(Pc.var(ddof=1) / Pc.size + Pa.var(ddof=1) / Pa.size)
    assert abs(Pc.mean() - Pa.mean()) < K_SE * se
    # second moments of the linear observable agree too (same Gaussian-like law)
    vc, va = rp["Y_c"][:, 0].var(ddof=1), ra["Y_f"][:, 0].var(ddof=1)
    assert abs(math.log(vc / va)) < K_SE * math.sqrt(2.0 / 1999 * 2)


def test_cross_level_variance_decays_at_high_density():
    N = 1e8
    levels = oracle.level_table(1.0, 8, 2, 0.005, 0.1)
    V = []
    for l in (1, 2):
        ol = _inputs(levels, N, _sinsin, _cos1, l, coupled=True)
        r = oracle.run_samples(ol, seed=31, ids=range(600), coupled=True)
        lf, lc = levels[l], levels[l - 1]
        Ybf = oracle.inner_h(oracle.mean_field(lf.n, lf.h, lf.tau, lf.M, _sinsin(lf.n)), _cos1(lf.n), lf.h)
        Ybc = oracle.inner_h(oracle.mean_field(lc.n, lc.h, lc.tau, lc.M, _sinsin(lc.n)), _cos1(lc.n), lc.h)
        dP = (oracle.observable_P(N, r["Y_f"], [Ybf]) - oracle.observable_P(N, r["Y_c"], [Ybc]))[:, 0]
        Pf = oracle.observable_P(N, r["Y_f"], [Ybf])[:, 0]
        V.append(dP.var(ddof=1))
        assert V[-1] < 0.2 * Pf.var(ddof=1)     # coupling removes most of the variance
    ratio = V[0] / V[1]
    assert 2.0 < ratio < 8.0                     # ~ h^2 decay for NN coupling (beta = 2)


# ----------------------------------------------------- Algorithm 1 host logic
def test_optimal_allocation_is_the_constrained_optimum():
    """Eq. (opt_M_ell) minimises sum M_l C_l subject to sum V_l / M_l = eps^2 / 2."""
    V = [0.3, 0.02, 4e-3, 9e-4]
    C = [1.0, 8.0, 64.0, 512.0]
    eps = 1e-3
    M = oracle.mlmc_optimal_samples(V, C, eps)
    # continuous optimum meets the variance budget with equality; ceil keeps it below
    assert sum(v / m for v, m in zip(V, M)) <= eps * eps / 2 * (1 + 1e-12)
    Mc = np.array([2 / eps ** 2 * math.sqrt(v / c) * sum(math.sqrt(a * b) for a, b in zip(V, C)) for v, c in zip(V, C)])
    assert sum(v / m for v, m in zip(V, Mc)) == pytest.approx(eps * eps / 2, rel=1e-12)
    cost = float(np.dot(Mc, C))
    rng = np.random.default_rng(0)
    for _ in range(200):
        w = np.exp(rng.normal(0, 0.3, size=len(V)))
        Mp = Mc * w
        Mp *= sum(v / m for v, m in zip(V, Mp)) / (eps * eps / 2)   # rescale onto the constraint
        assert float(np.dot(Mp, C)) >= cost * (1 - 1e-12)


def test_convergence_test_as_printed():
    eps = 1e-2
    lim = eps / math.sqrt(2) * 3.0     # (2^alpha - 1) eps / sqrt 2 with alpha = 2
    assert oracle.mlmc_converged([1.0, 0.5 * lim, 0.9 * lim, 0.9 * lim], eps) is True
    assert oracle.mlmc_converged([1.0, 0.5 * lim, 0.1, 0.9 * lim], eps) is False   # 0.1/4 > lim
    assert oracle.mlmc_converged([1.0, 0.5 * lim, 1.01 * lim * 4, 0.5 * lim], eps) is False
    assert oracle.mlmc_converged([1.0, 17 * lim, 0.9 * lim * 4, 0.5 * lim], eps) is False  # 17/16 > 1
    assert oracle.mlmc_converged([1.0, 15 * lim, 0.9 * lim * 4, 0.5 * lim], eps) is True
