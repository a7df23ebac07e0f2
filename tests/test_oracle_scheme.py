"""Deterministic pins for the oracle's scheme (Eq. FullyDiscreteDK with
b0 = 0, b1 = 1; operators of Section 7.2; NN coupling of Section 3.2).

Each check comes from outside the oracle's own code path: discrete Fourier
analysis (closed-form mode decay, FFT mean field), the textbook stability
limit of explicit 2-D heat stepping, exact conservation of the divergence
form, summation by parts for the one-step noise term, and an independent
dense-matrix restatement of the coupled pair on an 8 x 8 grid.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _grid(n, L):
    x = np.arange(n) * (L / n)
    return np.meshgrid(x, x, indexing="ij")


# --------------------------------------------------------------- mean field
@pytest.mark.parametrize("k", [(1, 0), (0, 1), (1, 1), (2, 3), (4, 4)])
@pytest.mark.parametrize("L", [1.0, 2 * math.pi])
def test_noise_off_mode_decays_by_discrete_symbol(k, L):
    n, M, mu = 16, 37, 0.2
    h = L / n
    tau = mu * h * h
    x1, x2 = _grid(n, L)
    w = 2 * math.pi / L
    mode_c = np.cos(w * (k[0] * x1 + k[1] * x2))
    mode_s = np.sin(w * (k[0] * x1 + k[1] * x2))
    rho0 = 1.0 + 0.3 * mode_c - 0.2 * mode_s
    out = oracle.mean_field(n, h, tau, M, rho0)
    # Delta_h on exp(i w k.x) has eigenvalue -4 (sin^2(pi k1/n) + sin^2(pi k2/n)) / h^2
    g = 1.0 - 2.0 * mu * (math.sin(math.pi * k[0] / n) ** 2 + math.sin(math.pi * k[1] / n) ** 2)
    expect = 1.0 + g ** M * (0.3 * mode_c - 0.2 * mode_s)
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-13)


def test_noise_off_sample_is_mean_field_and_matches_fft():
    n, L, mu, M = 16, 1.0, 0.15, 40
    h = L / n
    tau = mu * h * h
    x1, x2 = _grid(n, L)
    rho0 = 0.02 + np.exp(-((x1 - 0.3) ** 2 + (x2 - 0.6) ** 2) / 0.02)
    lv = oracle.Level(0, n, h, tau, M)
    ol = oracle.OracleLevel(lv, 0.0, rho0, [np.cos(2 * math.pi * x1)])
    r = ol.sample(seed=5, sample=3, coupled=False, fields=True)
    # library FFT diagonalises the circulant noise-free operator
    kk = np.fft.fftfreq(n) * n
    g = 1.0 - 2.0 * mu * (np.sin(math.pi * kk[:, None] / n) ** 2 + np.sin(math.pi * kk[None, :] / n) ** 2)
    fft_mf = np.real(np.fft.ifft2(np.fft.fft2(rho0) * g ** M))
    np.testing.assert_allclose(r["rho_f"], fft_mf, rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.mean_field(n, h, tau, M, rho0), fft_mf, rtol=0, atol=1e-12)


@pytest.mark.parametrize("mu,grows", [(0.24, False), (0.5, False), (0.52, True)])
def test_checkerboard_stability_limit(mu, grows):
    """Explicit 1/2 Delta_h stepping in 2-D is stable iff tau/h^2 <= 1/2: the
    checkerboard mode has symbol 1 - 4 mu (Assumption ass_stability)."""
    n, M = 8, 60
    h = 1.0 / n
    i1, i2 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    rho0 = 1e-3 * (-1.0) ** (i1 + i2)        # the scheme is linear: no offset needed
    out = oracle.mean_field(n, h, mu * h * h, M, rho0)
    amp = np.max(np.abs(out))
    assert amp == pytest.approx(1e-3 * abs(1 - 4 * mu) ** M, rel=1e-9, abs=1e-300)
    assert (amp > 1e-3) == grows


# --------------------------------------------------------------- noise term
def test_mass_conserved_exactly_with_noise_and_positive_part():
    """Sum_x Delta_h a = 0 and sum_x nabla_h . b = 0 on the torus, so the mass
    (rho, 1)_h is invariant even when [rho]^+ truncates (low density)."""
    n, L = 16, 1.0
    x1, x2 = _grid(n, L)
    rho0 = 0.02 + 0.98 * np.exp(-((x1 - 0.5) ** 2 + (x2 - 0.5) ** 2) / 0.02)
    lv = oracle.Level(2, n, L / n, 0.1 * (L / n) ** 2, 64)
    ol = oracle.OracleLevel(lv, 50.0, rho0, [np.ones_like(x1)], rho0[::2, ::2], [np.ones((8, 8))])
    r = ol.sample(seed=11, sample=0, coupled=True, fields=True)
    assert np.min(r["rho_f"]) < 0.0          # the positive part is active
    m0f = oracle.inner_h(rho0, np.ones_like(rho0), lv.h)
    m0c = oracle.inner_h(rho0[::2, ::2], np.ones((8, 8)), 2 * lv.h)
    assert r["mass_f"] == pytest.approx(m0f, rel=0, abs=1e-13)
    assert r["mass_c"] == pytest.approx(m0c, rel=0, abs=1e-13)


@pytest.mark.parametrize("k", [(1, 0), (1, 2)])
def test_one_step_noise_by_summation_by_parts(k):
    """After one step from deterministic rho0, Y - Ybar = N^-1/2 (nabla_h.b, phi)_h
    = -N^-1/2 (b, nabla^c_h phi)_h with b_r(y) = h^{-1} sqrt(rho0(y)^+) sqrt(tau) Z_(y,r)."""
    n, L, N = 16, 1.0, 1e3
    h = L / n
    tau = 0.1 * h * h
    x1, x2 = _grid(n, L)
    rho0 = 1.0 + 0.5 * np.sin(2 * math.pi * x1) * np.sin(2 * math.pi * x2)
    phi = np.cos(2 * math.pi * (k[0] * x1 + k[1] * x2))
    lv = oracle.Level(1, n, h, tau, 1)
    ol = oracle.OracleLevel(lv, N, rho0, [phi])
    seed, s = 9, 4
    Y = ol.sample(seed, s, coupled=False)["Y_f"][0]
    Ybar = oracle.inner_h(oracle.mean_field(n, h, tau, 1, rho0), phi, h)
    Z = oracle.normals(seed, 1, 0, s, 0, n)
    grad1 = (np.roll(phi, -1, 0) - np.roll(phi, 1, 0)) / (2 * h)
    grad2 = (np.roll(phi, -1, 1) - np.roll(phi, 1, 1)) / (2 * h)
    b1 = np.sqrt(rho0) * math.sqrt(tau) * Z[..., 0] / h
    b2 = np.sqrt(rho0) * math.sqrt(tau) * Z[..., 1] / h
    expect = -(h * h) * np.sum(b1 * grad1 + b2 * grad2) / math.sqrt(N)
    assert Y - Ybar == pytest.approx(expect, rel=1e-11, abs=1e-17)


# ----------------------------------------------------- 8x8 brute force pair
def _dense_operators(n, h):
    """Dense periodic 5-point Laplacian and central-difference divergence."""
    idx = lambda i1, i2: (i1 % n) * n + (i2 % n)
    Lap = np.zeros((n * n, n * n))
    D1 = np.zeros((n * n, n * n))
    D2 = np.zeros((n * n, n * n))
    for i1 in range(n):
        for i2 in range(n):
            x = idx(i1, i2)
            Lap[x, x] -= 4 / h ** 2
            for y in (idx(i1 + 1, i2), idx(i1 - 1, i2), idx(i1, i2 + 1), idx(i1, i2 - 1)):
                Lap[x, y] += 1 / h ** 2
            D1[x, idx(i1 + 1, i2)] += 1 / (2 * h)
            D1[x, idx(i1 - 1, i2)] -= 1 / (2 * h)
            D2[x, idx(i1, i2 + 1)] += 1 / (2 * h)
            D2[x, idx(i1, i2 - 1)] -= 1 / (2 * h)
    return Lap, D1, D2


def test_brute_force_8x8_coupled_pair():
    n, nc, L, N, M = 8, 4, 1.0, 30.0, 16
    h = L / n
    tau = 0.12 * h * h
    x1, x2 = _grid(n, L)
    rho0 = 1.0 + 0.5 * np.sin(2 * math.pi * x1) * np.sin(2 * math.pi * x2) + 0.3 * np.cos(4 * math.pi * x2)
    rho0c = rho0[::2, ::2]
    phi = np.cos(2 * math.pi * x1)
    lv = oracle.Level(1, n, h, tau, M)
    ol = oracle.OracleLevel(lv, N, rho0, [phi], rho0c, [phi[::2, ::2]])
    seed, s = 21, 2
    r = ol.sample(seed, s, coupled=True, fields=True)

    Lap, D1, D2 = _dense_operators(n, h)
    Lapc, D1c, D2c = _dense_operators(nc, 2 * h)
    # coupling matrix: coarse BM = 2^{-1} x sum of the fine BMs at y + h v, v in {0,1}^2
    B = np.zeros((nc * nc, n * n))
    for I1 in range(nc):
        for I2 in range(nc):
            for v1 in (0, 1):
                for v2 in (0, 1):
                    B[I1 * nc + I2, (2 * I1 + v1) * n + (2 * I2 + v2)] = 0.5
    rf = rho0.reshape(-1).copy()
    rc = rho0c.reshape(-1).copy()
    acc = np.zeros((nc * nc, 2))
    for m in range(M):
        Z = oracle.normals(seed, 1, 0, s, m, n).reshape(-1, 2)
        db = math.sqrt(tau) * Z
        acc += B @ db
        sq = np.sqrt(np.maximum(rf, 0))
        rf = rf + 0.5 * tau * (Lap @ rf) + (D1 @ (sq * db[:, 0] / h) + D2 @ (sq * db[:, 1] / h)) / math.sqrt(N)
        if m % 4 == 3:
            sqc = np.sqrt(np.maximum(rc, 0))
            hc = 2 * h
            rc = rc + 0.5 * (4 * tau) * (Lapc @ rc) + (D1c @ (sqc * acc[:, 0] / hc) + D2c @ (sqc * acc[:, 1] / hc)) / math.sqrt(N)
            acc[:] = 0
    np.testing.assert_allclose(r["rho_f"].reshape(-1), rf, rtol=0, atol=1e-13)
    np.testing.assert_allclose(r["rho_c"].reshape(-1), rc, rtol=0, atol=1e-13)
    assert r["Y_f"][0] == pytest.approx(h * h * np.sum(rf * phi.reshape(-1)), abs=1e-14)
    assert r["Y_c"][0] == pytest.approx(4 * h * h * np.sum(rc * phi[::2, ::2].reshape(-1)), abs=1e-14)


def test_coarse_increment_is_standard_brownian():
    """Each coarse increment 1/2 sum_{v} sum_{j<4} dbeta_fine has variance
    4 tau = tau_{l-1} (Remark distribution_W_ell, NN form): check on the
    normals the coupling sums."""
    n, seed = 64, 4
    acc = np.zeros((n // 2, n // 2, 2))
    for m in range(4):
        Z = oracle.normals(seed, 3, 0, 17, m, n)
        acc += 0.5 * (Z[0::2, 0::2] + Z[1::2, 0::2] + Z[0::2, 1::2] + Z[1::2, 1::2])
    z = acc.reshape(-1) / 2.0      # dbeta_c / sqrt(tau_c) with tau_c = 4 tau
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)


# ------------------------------------------------------ level hierarchy pin
def test_level_table_reproduces_paper_setting():
    g = json.load(open(os.path.join(HERE, "golden", "paper_level_hierarchy.json")))
    lt = oracle.level_table(g["length"], 4, g["L_max"], g["T"], mu=0.0, M0=1)
    for ref, lv in zip(g["levels"], lt):
        assert lv.n == ref["cells_per_axis"]
        assert lv.h == pytest.approx(ref["h"], rel=1e-15)
        assert lv.tau == pytest.approx(ref["tau"], rel=1e-14)
        assert lv.M * lv.tau == pytest.approx(g["T"], rel=1e-14)
        assert lv.tau / lv.h ** 2 == pytest.approx(lt[0].tau / lt[0].h ** 2, rel=1e-13)


def test_level_table_rounds_steps_up_and_keeps_cfl():
    lt = oracle.level_table(1.0, 16, 4, 0.02, 0.1)
    assert [lv.M for lv in lt] == [52, 208, 832, 3328, 13312]
    for lv in lt:
        assert lv.tau / lv.h ** 2 <= 0.1
        assert lv.M * lv.tau == pytest.approx(0.02, rel=1e-14)
    assert oracle.level_table(1.0, 32, 0, 0.01, 0.1)[0].M == 103
    assert oracle.level_table(1.0, 32, 5, 0.05, 0.1)[0].M == 512
