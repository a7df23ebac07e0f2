"""Pins for the oracle's Fourier coupling (Section 3.1: h_{l-1} = 3 h_l,
tau_{l-1} = 9 tau_l; the coarse noise carries every Fourier mode of the fine
noise that the coarse grid resolves, summed over the 9 fine steps of a coarse
step).

Checked from outside the oracle's code path: numpy FFTs of its coarse field
against those of the fine field (shared modes equal, the Nyquist alias pair
combined), the restriction as a matrix (rows orthonormal, so white noise stays
white with the same variance: Remark distribution_W_ell), resolved smooth
modes carried unchanged, a dense restatement of a whole coupled pair on a
6 x 6 / 2 x 2 grid built from numpy's complex exponentials, the law of the
coarse member against stand-alone coarse paths on seeded samples, and
E[Y] = Ybar on both members at low density.
"""
import math

import numpy as np
import pytest

import oracle


def _grid(n, L=1.0):
    x = np.arange(n) * (L / n)
    return np.meshgrid(x, x, indexing="ij")


@pytest.mark.parametrize("n", [6, 18, 54, 162])
def test_shared_modes_are_the_fine_modes(n):
    nc = n // 3
    K = nc // 2
    f = np.random.default_rng(n).standard_normal((n, n))
    g = oracle.fourier_restrict(n, nc, f)
    cf = np.fft.fft2(f) / n          # unitary coefficients
    cg = np.fft.fft2(g) / nc
    for a in range(-K + 1, K):
        for b in range(-K + 1, K):
            assert abs(cg[a % nc, b % nc] - cf[a % n, b % n]) < 1e-12
    # the coarse Nyquist mode along axis 1 takes the two fine aliases with weight 2^-1/2 each
    for b in range(-K + 1, K):
        expect = (cf[-K % n, b % n] + cf[K % n, b % n]) / math.sqrt(2.0)
        assert abs(cg[K % nc, b % nc] - expect) < 1e-12


@pytest.mark.parametrize("n", [6, 18])
def test_restriction_rows_are_orthonormal(n):
    """As a matrix on fine fields the restriction has orthonormal rows: a white
    fine field gives a white coarse field of the same variance."""
    nc = n // 3
    P = np.stack([oracle.fourier_restrict(n, nc, e.reshape(n, n)).reshape(-1) for e in np.eye(n * n)], axis=1)
    np.testing.assert_allclose(P @ P.T, np.eye(nc * nc), rtol=0, atol=1e-13)


@pytest.mark.parametrize("k", [(1, 0), (2, 1), (0, 2)])
def test_resolved_smooth_mode_is_carried_unchanged(k):
    """A mode the coarse grid resolves reaches it with the fine noise's
    amplitude per unit of h^-1: coarse values = 3 x fine values (h_c = 3 h)."""
    n, nc = 18, 6
    x1, x2 = _grid(n)
    y1, y2 = _grid(nc)
    f = np.cos(2 * math.pi * (k[0] * x1 + k[1] * x2)) + 0.5 * np.sin(2 * math.pi * (k[0] * x1 + k[1] * x2))
    g = np.cos(2 * math.pi * (k[0] * y1 + k[1] * y2)) + 0.5 * np.sin(2 * math.pi * (k[0] * y1 + k[1] * y2))
    np.testing.assert_allclose(oracle.fourier_restrict(n, nc, f), 3.0 * g, rtol=0, atol=1e-12)


def _restriction_1d(n, nc):
    """P1[y, x] = (n nc)^-1/2 sum_{xi=-K..K} w(xi) exp(2 pi i xi (y/nc - x/n)), real."""
    K = nc // 2
    P = np.zeros((nc, n), dtype=complex)
    for xi in range(-K, K + 1):
        w = 1 / math.sqrt(2) if abs(xi) == K else 1.0
        P += w * np.exp(2j * math.pi * xi * (np.arange(nc)[:, None] / nc - np.arange(n)[None, :] / n))
    assert np.max(np.abs(P.imag)) < 1e-12
    return P.real / math.sqrt(n * nc)


def _dense(n, h):
    idx = lambda i1, i2: (i1 % n) * n + (i2 % n)
    Lap, D1, D2 = (np.zeros((n * n, n * n)) for _ in range(3))
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


def test_brute_force_fourier_pair_6x6():
    n, nc, N, M = 6, 2, 40.0, 18
    h = 1.0 / n
    tau = 0.1 * h * h
    x1, x2 = _grid(n)
    rho0 = 1.0 + 0.5 * np.sin(2 * math.pi * x1) * np.sin(2 * math.pi * x2) + 0.2 * np.cos(2 * math.pi * x2)
    rho0c = rho0[::3, ::3]
    phi = np.cos(2 * math.pi * x1)
    lv = oracle.Level(1, n, h, tau, M)
    ol = oracle.OracleLevel(lv, N, rho0, [phi], rho0c, [phi[::3, ::3]], coupling=1)
    seed, s = 5, 7
    r = ol.sample(seed, s, coupled=True, fields=True)
    P1 = _restriction_1d(n, nc)
    Lap, D1, D2 = _dense(n, h)
    Lc, D1c, D2c = _dense(nc, 3 * h)
    rf = rho0.reshape(-1).copy()
    rc = rho0c.reshape(-1).copy()
    acc = np.zeros((n, n, 2))
    for m in range(M):
        db = math.sqrt(tau) * oracle.normals(seed, 1, 0, s, m, n)
        acc += db
        sq = np.sqrt(np.maximum(rf, 0))
        rf = rf + 0.5 * tau * (Lap @ rf) + (D1 @ (sq * db[..., 0].reshape(-1) / h) +
                                            D2 @ (sq * db[..., 1].reshape(-1) / h)) / math.sqrt(N)
        if m % 9 == 8:
            dbc = [(P1 @ acc[..., c] @ P1.T).reshape(-1) for c in range(2)]
            sqc = np.sqrt(np.maximum(rc, 0))
            hc = 3 * h
            rc = rc + 0.5 * (9 * tau) * (Lc @ rc) + (D1c @ (sqc * dbc[0] / hc) + D2c @ (sqc * dbc[1] / hc)) / math.sqrt(N)
            acc[:] = 0
    np.testing.assert_allclose(r["rho_f"].reshape(-1), rf, rtol=0, atol=1e-13)
    np.testing.assert_allclose(r["rho_c"].reshape(-1), rc, rtol=0, atol=1e-13)


def test_level_table_ratio_three():
    lv = oracle.level_table(1.0, 6, 2, 0.02, 0.1, ratio=3)
    assert [l.n for l in lv] == [6, 18, 54]
    assert [l.M for l in lv] == [8, 72, 648]
    assert all(abs(l.tau / l.h ** 2 - lv[0].tau / lv[0].h ** 2) < 1e-12 for l in lv)


def test_coarse_member_has_law_of_standalone_coarse_path():
    """Remark distribution_W_ell for the Fourier coupling: the coarse member of
    a level-1 pair has the law of a level-0 path (mean and variance of P)."""
    N = 2e3
    levels = oracle.level_table(1.0, 6, 1, 0.02, 0.1, ratio=3)
    rho = lambda n: 1.0 + 0.5 * np.sin(2 * math.pi * _grid(n)[0]) * np.sin(2 * math.pi * _grid(n)[1])
    phi = lambda n: np.cos(2 * math.pi * _grid(n)[0])
    pair = oracle.OracleLevel(levels[1], N, rho(18), [phi(18)], rho(6), [phi(6)], coupling=1)
    alone = oracle.OracleLevel(levels[0], N, rho(6), [phi(6)], coupling=1)
    lc = levels[0]
    ybar = oracle.inner_h(oracle.mean_field(6, lc.h, lc.tau, lc.M, rho(6)), phi(6), lc.h)
    yc = oracle.run_samples(pair, 3, range(3000), True)["Y_c"][:, 0]
    ya = oracle.run_samples(alone, 4, range(3000), False, stream=1)["Y_f"][:, 0]
    pc, pa = N * (yc - ybar) ** 2, N * (ya - ybar) ** 2
    se = math.sqrt(pc.var(ddof=1) / pc.size + pa.var(ddof=1) / pa.size)
    assert abs(pc.mean() - pa.mean()) < 3.5 * se
    # variances of P within sampling error (ratio of variances, F-distribution spread ~ 2/sqrt(n))
    assert abs(pc.var() / pa.var() - 1.0) < 0.2


def test_mean_of_Y_is_the_mean_field_on_both_members():
    """E[Y_f] = Ybar_l and E[Y_c] = Ybar_{l-1} for Fourier-coupled pairs at low
    density (the restricted noise has zero mean)."""
    N = 50.0
    levels = oracle.level_table(1.0, 6, 1, 0.02, 0.1, ratio=3)
    g = lambda n: 0.05 + np.exp(-((_grid(n)[0] - 0.5) ** 2 + (_grid(n)[1] - 0.5) ** 2) / 0.05)
    phi = lambda n: np.cos(2 * math.pi * _grid(n)[0])
    ol = oracle.OracleLevel(levels[1], N, g(18), [phi(18)], g(6), [phi(6)], coupling=1)
    r = oracle.run_samples(ol, 6, range(2000), True)
    for key, lv in (("Y_f", levels[1]), ("Y_c", levels[0])):
        ybar = oracle.inner_h(oracle.mean_field(lv.n, lv.h, lv.tau, lv.M, g(lv.n)), phi(lv.n), lv.h)
        y = r[key][:, 0]
        assert abs(y.mean() - ybar) < 3.5 * y.std(ddof=1) / math.sqrt(y.size), key
