"""Pins for the surrogate oracle (FP64): orthonormal modes, the exact Gaussian
law of the heat-weighted features, and the MLP gradient against central finite
differences."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import surrogate as sg


@pytest.mark.parametrize("n", [8, 16, 32])
def test_modes_are_orthonormal_and_lowest(n):
    E = sg.modes(n, 32).reshape(32, -1)
    np.testing.assert_allclose(E @ E.T, np.eye(32), atol=1e-12)
    ks = sg.mode_vectors(n, 32)
    k2 = [a * a + b * b for a, b in ks]
    assert k2 == sorted(k2) and k2[0] == 1 and max(k2) <= 10


def test_heat_factors_are_the_scheme_symbol():
    n, mu = 16, 0.0985
    g = sg.heat_factors(n, mu)
    E = sg.modes(n)
    h = 1.0 / n
    for j in (0, 5, 17):
        rho = E[j].copy()
        one = oracle.dk_step(n, h, mu * h * h, 0.0, rho, None)
        np.testing.assert_allclose(one, g[j] * rho, atol=1e-14)


def test_features_have_the_exact_gaussian_law():
    n, M, mu = 16, 13, 0.0985
    E, g = sg.modes(n), sg.heat_factors(n, mu)
    sig = sg.feature_sigma(g, M)
    X = []
    for s in range(600):
        Zs = [oracle.normals(7, 0, 3, s, m, n) for m in range(M)]
        X.append(sg.features(Zs, E, g) / sig)
    X = np.array(X)
    flat = X.reshape(-1)
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    C = np.corrcoef(X.T)
    off = C[~np.eye(64, dtype=bool)]
    assert np.max(np.abs(off)) < 5.0 / math.sqrt(600)
    assert abs(flat.var() - 1.0) < 5 * math.sqrt(2.0 / flat.size)


@pytest.mark.parametrize("outputs", [1, 4])
def test_mlp_gradient_matches_finite_differences(outputs):
    rng = np.random.default_rng(0)
    P = sg.mlp_param_count(outputs)
    assert P == 148224 + 257 * outputs     # 64*256+256 + 2*(256*256+256) + (256+1)*K
    theta = rng.normal(0, 0.08, size=P)
    X = rng.normal(size=(16, 64))
    T = rng.normal(size=16) if outputs == 1 else rng.normal(size=(16, outputs))
    loss, grad = sg.mlp_loss_grad(theta, X, T)
    idx = rng.choice(P, size=60, replace=False)
    for i in idx:
        e = np.zeros(P)
        e[i] = 1e-6
        lp, _ = sg.mlp_loss_grad(theta + e, X, T)
        lm, _ = sg.mlp_loss_grad(theta - e, X, T)
        fd = (lp - lm) / 2e-6
        assert fd == pytest.approx(grad[i], rel=1e-5, abs=1e-9)
