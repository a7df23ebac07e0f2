"""Pins for the oracle's theta-scheme: Eq. (FullyDiscreteDK) with weights
b0 > 0, b1 = 1 - b0 (Definition 2.1; the operator A_h of Appendix C,
Lemma Discrete_Energy_Est).

The oracle solves the periodic system (I - b0 tau/2 Delta_h) rho^m = rhs by
discrete Fourier diagonalisation.  Each check below comes from outside that
code path: the linear system itself applied with shifted arrays (residual),
a dense LU solve on 8 x 8 grids (one step and a whole coupled pair), the
special case b0 = 0 (the explicit oracle), the mode symbol
(1 - b1 lam)/(1 + b0 lam), the stability threshold it implies, exact mass
conservation, the martingale closed form of E[P] (with the factor the
solve puts on the noise) on seeded samples, and E[Y] = Ybar at low density.
"""
import math

import numpy as np
import pytest

import oracle


def _grid(n, L=1.0):
    x = np.arange(n) * (L / n)
    return np.meshgrid(x, x, indexing="ij")


def _lap(a, h):
    """Delta_h a with the 5-point stencil of Section 7.2 (periodic)."""
    return (np.roll(a, 1, 0) + np.roll(a, -1, 0) + np.roll(a, 1, 1) + np.roll(a, -1, 1) - 4.0 * a) / (h * h)


def _noise_div(rho, dbeta, h, inv_sqrt_N):
    """inv_sqrt_N nabla_h . (h^-1 sqrt([rho]^+) dbeta), central differences."""
    s = np.sqrt(np.maximum(rho, 0.0))
    F1 = s * dbeta[..., 0] / h
    F2 = s * dbeta[..., 1] / h
    div = (np.roll(F1, -1, 0) - np.roll(F1, 1, 0)) / (2 * h) + (np.roll(F2, -1, 1) - np.roll(F2, 1, 1)) / (2 * h)
    return inv_sqrt_N * div


def _state(n, seed):
    rng = np.random.default_rng(seed)
    x1, x2 = _grid(n)
    rho = 1.0 + 0.5 * np.sin(2 * math.pi * x1) * np.sin(2 * math.pi * x2) + 0.05 * rng.standard_normal((n, n))
    rho[0, 0] = -0.1     # one cell below 0: the positive part is active
    return rho, rng.standard_normal((n, n, 2))


def test_b0_zero_is_the_explicit_step():
    n, h = 16, 1.0 / 16
    tau = 0.2 * h * h
    rho, Z = _state(n, 1)
    db = math.sqrt(tau) * Z
    a = oracle.theta_step(n, h, tau, 0.01, 0.0, rho, db)
    b = oracle.dk_step(n, h, tau, 0.01, rho, db)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("b0,mu", [(0.5, 0.4), (0.5, 3.0), (1.0, 1.0), (0.3, 0.9)])
def test_step_satisfies_its_linear_system(b0, mu):
    """(I - b0 tau/2 Delta_h) out - (I + b1 tau/2 Delta_h) rho - xi = 0 with
    Delta_h and nabla_h applied by array shifts, not by the Fourier solve."""
    n = 16
    h = 1.0 / n
    tau = mu * h * h
    rho, Z = _state(n, 2)
    db = math.sqrt(tau) * Z
    out = oracle.theta_step(n, h, tau, 0.03, b0, rho, db)
    lhs = out - b0 * 0.5 * tau * _lap(out, h)
    rhs = rho + (1.0 - b0) * 0.5 * tau * _lap(rho, h) + _noise_div(rho, db, h, 0.03)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-13 * (1 + mu))


def _dense_L(n):
    """L = -h^2 Delta_h as a dense matrix on the flattened periodic grid."""
    Lm = np.zeros((n * n, n * n))
    for i1 in range(n):
        for i2 in range(n):
            x = i1 * n + i2
            Lm[x, x] = 4.0
            for j1, j2 in ((i1 + 1, i2), (i1 - 1, i2), (i1, i2 + 1), (i1, i2 - 1)):
                Lm[x, (j1 % n) * n + (j2 % n)] -= 1.0
    return Lm


@pytest.mark.parametrize("c", [0.0, 0.05, 0.7, 12.0])
def test_helmholtz_solve_against_dense_lu(c):
    n = 8
    rhs = np.random.default_rng(3).standard_normal((n, n))
    expect = np.linalg.solve(np.eye(n * n) + c * _dense_L(n), rhs.reshape(-1)).reshape(n, n)
    np.testing.assert_allclose(oracle.helmholtz_solve(n, c, rhs), expect, rtol=0, atol=1e-13)


@pytest.mark.parametrize("b0", [0.5, 1.0])
@pytest.mark.parametrize("k", [(1, 0), (2, 3), (4, 4)])
def test_noise_off_mode_decays_by_theta_symbol(b0, k):
    n, M, mu = 16, 23, 1.5
    h = 1.0 / n
    x1, x2 = _grid(n)
    arg = 2 * math.pi * (k[0] * x1 + k[1] * x2)
    rho0 = 1.0 + 0.3 * np.cos(arg) - 0.2 * np.sin(arg)
    out = oracle.mean_field(n, h, mu * h * h, M, rho0, b0=b0)
    lam = 2.0 * mu * (math.sin(math.pi * k[0] / n) ** 2 + math.sin(math.pi * k[1] / n) ** 2)
    g = (1.0 - (1.0 - b0) * lam) / (1.0 + b0 * lam)
    assert g == pytest.approx(oracle.heat_symbol(k, n, mu, b0), rel=1e-15)
    np.testing.assert_allclose(out, 1.0 + g ** M * (0.3 * np.cos(arg) - 0.2 * np.sin(arg)), rtol=0, atol=1e-13)


@pytest.mark.parametrize("b0,mu,grows", [(0.25, 0.99, False), (0.25, 1.01, True), (0.5, 50.0, False),
                                         (1.0, 50.0, False)])
def test_checkerboard_stability_threshold(b0, mu, grows):
    """The checkerboard mode has lam = 4 mu: |g| <= 1 iff (b1 - b0) 2 mu <= 1,
    so b0 >= 1/2 is stable for every tau/h^2 (Assumption ass_stability)."""
    n, M = 8, 80
    h = 1.0 / n
    i1, i2 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    rho0 = 1e-3 * (-1.0) ** (i1 + i2)
    amp = np.max(np.abs(oracle.mean_field(n, h, mu * h * h, M, rho0, b0=b0)))
    g = (1.0 - (1.0 - b0) * 4 * mu) / (1.0 + b0 * 4 * mu)
    # the Fourier solve leaves rounding of ~1e-19 x 1e-3 in the other modes
    assert amp == pytest.approx(1e-3 * abs(g) ** M, rel=1e-9, abs=1e-18)
    assert (amp > 1e-3) == grows


def test_mass_conserved_with_noise_and_positive_part():
    n = 16
    h = 1.0 / n
    x1, x2 = _grid(n)
    rho0 = 0.02 + 0.98 * np.exp(-((x1 - 0.5) ** 2 + (x2 - 0.5) ** 2) / 0.02)
    lv = oracle.Level(2, n, h, 1.2 * h * h, 32)
    ol = oracle.OracleLevel(lv, 50.0, rho0, [np.ones_like(x1)], rho0[::2, ::2], [np.ones((8, 8))], b0=0.5)
    r = ol.sample(seed=11, sample=0, coupled=True, fields=True)
    assert np.min(r["rho_f"]) < 0.0
    assert r["mass_f"] == pytest.approx(oracle.inner_h(rho0, np.ones_like(rho0), h), rel=0, abs=1e-13)
    assert r["mass_c"] == pytest.approx(oracle.inner_h(rho0[::2, ::2], np.ones((8, 8)), 2 * h), rel=0, abs=1e-13)


@pytest.mark.parametrize("b0", [0.5, 1.0])
def test_brute_force_8x8_coupled_pair(b0):
    """The coupled pair restated with dense matrices and LU solves."""
    n, nc, N, M = 8, 4, 30.0, 16
    h = 1.0 / n
    tau = 0.9 * h * h
    x1, x2 = _grid(n)
    rho0 = 1.0 + 0.5 * np.sin(2 * math.pi * x1) * np.sin(2 * math.pi * x2) + 0.3 * np.cos(4 * math.pi * x2)
    rho0c = rho0[::2, ::2]
    phi = np.cos(2 * math.pi * x1)
    lv = oracle.Level(1, n, h, tau, M)
    ol = oracle.OracleLevel(lv, N, rho0, [phi], rho0c, [phi[::2, ::2]], b0=b0)
    seed, s = 21, 2
    r = ol.sample(seed, s, coupled=True, fields=True)

    def dense_step(nn, hh, tt, rho, db):
        Lm = _dense_L(nn) / (hh * hh)          # -Delta_h
        rhs = rho + (1.0 - b0) * 0.5 * tt * (-Lm @ rho)
        rhs = rhs + _noise_div(rho.reshape(nn, nn), db.reshape(nn, nn, 2), hh, 1 / math.sqrt(N)).reshape(-1)
        return np.linalg.solve(np.eye(nn * nn) + b0 * 0.5 * tt * Lm, rhs)

    rf = rho0.reshape(-1).copy()
    rc = rho0c.reshape(-1).copy()
    acc = np.zeros((nc, nc, 2))
    for m in range(M):
        db = math.sqrt(tau) * oracle.normals(seed, 1, 0, s, m, n)
        acc += 0.5 * db.reshape(nc, 2, nc, 2, 2).sum(axis=(1, 3))
        rf = dense_step(n, h, tau, rf, db)
        if m % 4 == 3:
            rc = dense_step(nc, 2 * h, 4 * tau, rc, acc)
            acc[:] = 0
    np.testing.assert_allclose(r["rho_f"].reshape(-1), rf, rtol=0, atol=1e-13)
    np.testing.assert_allclose(r["rho_c"].reshape(-1), rc, rtol=0, atol=1e-13)


@pytest.mark.parametrize("b0,mu", [(0.5, 1.0), (1.0, 2.0)])
def test_mean_of_P_matches_martingale_closed_form(b0, mu):
    """E[P] with the solve's factor w^2 on the noise (rho stays positive)."""
    N, n, T = 1e8, 16, 0.02
    lv = oracle.level_table(1.0, n, 0, T, mu)[0]
    x1, x2 = _grid(n)
    rho0 = 1.0 + 0.5 * np.sin(2 * math.pi * x1) * np.sin(2 * math.pi * x2)
    phi = np.cos(2 * math.pi * x1)
    ol = oracle.OracleLevel(lv, N, rho0, [phi], b0=b0)
    r = oracle.run_samples(ol, seed=7, ids=range(2500), coupled=False, stream=1)
    Ybar = oracle.inner_h(oracle.mean_field(n, lv.h, lv.tau, lv.M, rho0, b0=b0), phi, lv.h)
    P = oracle.observable_P(N, r["Y_f"], [Ybar])[:, 0]
    se = P.std(ddof=1) / math.sqrt(P.size)
    expect = oracle.closed_form_EP_cos1(1.0, n, lv.tau, lv.M, b0=b0)
    assert abs(P.mean() - expect) < 3.5 * se
    assert se / expect < 0.05


def test_mean_of_Y_is_the_theta_mean_field_at_low_density():
    """E[Y] = Ybar for the theta-scheme too (linear scheme, zero-mean noise),
    even where [rho]^+ truncates."""
    N, n = 30.0, 8
    lv = oracle.level_table(1.0, n, 0, 0.02, 1.5)[0]
    x1, x2 = _grid(n)
    rho0 = 0.02 + np.exp(-((x1 - 0.5) ** 2 + (x2 - 0.5) ** 2) / 0.02)
    phi = np.cos(2 * math.pi * x1)
    ol = oracle.OracleLevel(lv, N, rho0, [phi], b0=0.5)
    y = oracle.run_samples(ol, seed=3, ids=range(3000), coupled=False, stream=1)["Y_f"][:, 0]
    ybar = oracle.inner_h(oracle.mean_field(n, lv.h, lv.tau, lv.M, rho0, b0=0.5), phi, lv.h)
    assert abs(y.mean() - ybar) < 3.5 * y.std(ddof=1) / math.sqrt(y.size)
