"""Learned level below level 0: GPU kernels against the FP64 surrogate oracle
(features, direct sampler, network forward and gradient), training, and the
unbiasedness of the surrogate-augmented estimator."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import surrogate as sg
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


def _bm(a, b):
    u = (a + 1.0) / 2.0 ** 32
    th = 2.0 * math.pi * (b + 0.5) / 2.0 ** 32
    r = math.sqrt(-2.0 * math.log(u))
    return r * math.cos(th), r * math.sin(th)


def test_features_match_oracle(dk):
    wl = W.get("mlmc16_256").with_(L_max=1)
    with dk.Context.from_workload(wl) as ctx:
        ctx.surrogate_init(1)
        info = ctx.level_info(0)
        X = ctx.surrogate_features(5, 6, seed=9, stream_tag=3)
    n, M = info.n, info.M
    mu = info.tau / info.h ** 2
    E, g = sg.modes(n), sg.heat_factors(n, mu)
    sig = sg.feature_sigma(g, M)
    for i in range(6):
        Zs = [oracle.normals(9, 0, 3, 5 + i, m, n) for m in range(M)]
        ref = sg.features(Zs, E, g) / sig
        np.testing.assert_allclose(X[i], ref, atol=2e-5, rtol=0)


def test_direct_features_are_the_philox_normals(dk):
    wl = W.get("mlmc16_256").with_(L_max=1)
    with dk.Context.from_workload(wl) as ctx:
        ctx.surrogate_init(1)
        X = ctx.surrogate_features(3, 4000, seed=12, stream_tag=2, direct=True)
    for s in (0, 1, 3999):
        sid = 3 + s
        for j in range(16):
            w = oracle.philox4x32_10([j, 0, sid, 0 | (2 << 8)], [12, 0])
            z = _bm(w[0], w[1]) + _bm(w[2], w[3])
            np.testing.assert_allclose(X[s, 4 * j:4 * j + 4], z, atol=5e-6 * 7, rtol=0)
    assert stats.kstest(X.reshape(-1), "norm").pvalue > 1e-3


def _bf16(a):
    """Round to BF16 (nearest, ties to even) and back, as the kernels store values."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _bf16_network(theta, X, T):
    """FP64 network that rounds to BF16 exactly where the GPU kernels store BF16
    (inputs, W1..W3, hidden activations and their gradients); FP32/FP64
    accumulation elsewhere.  T: (B,) or (B, K).  Returns (y, loss, flat gradient)."""
    T2 = T[:, None] if T.ndim == 1 else T
    K = T2.shape[1]
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = sg.mlp_unpack(theta.astype(np.float64), K)
    Xb = _bf16(X)
    W1b, W2b, W3b = _bf16(W1), _bf16(W2), _bf16(W3)
    H1 = _bf16(np.maximum(Xb @ W1b.T + b1, 0))
    H2 = _bf16(np.maximum(H1 @ W2b.T + b2, 0))
    H3 = _bf16(np.maximum(H2 @ W3b.T + b3, 0))
    y = H3 @ W4.T + b4
    B = X.shape[0]
    dy = 2.0 * (y - T2) / B
    loss = float(np.sum((y - T2) ** 2) / B)
    dH3 = _bf16((dy @ W4) * (H3 > 0))
    gW4, gb4 = dy.T @ H3, dy.sum(0)
    gW3, gb3 = dH3.T @ H2, dH3.sum(0)
    dH2 = _bf16((dH3 @ W3b) * (H2 > 0))
    gW2, gb2 = dH2.T @ H1, dH2.sum(0)
    dH1 = _bf16((dH2 @ W2b) * (H1 > 0))
    gW1, gb1 = dH1.T @ Xb, dH1.sum(0)
    grad = np.concatenate([gW1.reshape(-1), gb1, gW2.reshape(-1), gb2, gW3.reshape(-1), gb3, gW4.reshape(-1), gb4])
    return (y[:, 0] if T.ndim == 1 else y), loss, grad


@pytest.mark.parametrize("name,outputs", [("mlmc16_256", 1), ("large32_1024", 4)])
def test_forward_and_gradient_match_fp64_mlp(dk, name, outputs):
    """Against the BF16-rounding FP64 network: agreement to FP32-accumulation
    level; against the exact FP64 network (finite-difference pinned in the
    oracle tests): the BF16 bound, direction and size within a few percent.
    Four outputs: one per test function of the four-mode workload."""
    wl = W.get(name).with_(L_max=1)
    rng = np.random.default_rng(4)
    theta = rng.normal(0, 0.05, size=sg.mlp_param_count(outputs)).astype(np.float32)
    X = rng.normal(size=(512, 64)).astype(np.float32)
    T = (rng.normal(size=512) if outputs == 1 else rng.normal(size=(512, outputs))).astype(np.float32)
    with dk.Context.from_workload(wl) as ctx:
        ctx.surrogate_init(1)
        assert ctx.surrogate_info() == (sg.mlp_param_count(outputs), outputs)
        ctx.surrogate_params(theta)
        y = ctx.surrogate_forward(X)
        loss, grad = ctx.surrogate_loss_grad(X, T)
    y_b, loss_b, grad_b = _bf16_network(theta, X.astype(np.float64), T.astype(np.float64))
    err = np.abs(y - y_b)
    scale = np.max(np.abs(y_b))
    # FP32 vs FP64 accumulation for almost all rows; where a hidden activation sits
    # on a BF16 rounding boundary the two round it to neighbouring values, which
    # moves the output by about one BF16 step (2^-8) of that activation's share.
    assert np.median(err) <= 1e-6 * scale
    assert np.mean(err <= 1e-5 * scale) >= 0.95
    assert np.max(err) <= 2e-3 * scale
    assert loss == pytest.approx(loss_b, rel=1e-3)
    assert np.linalg.norm(grad - grad_b) <= 1e-2 * np.linalg.norm(grad_b)
    print("forward max/median err", err.max(), np.median(err), "grad rel err",
          np.linalg.norm(grad - grad_b) / np.linalg.norm(grad_b))
    _, grad_ref = sg.mlp_loss_grad(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert grad.shape == grad_ref.shape
    cos = float(np.dot(grad, grad_ref) / (np.linalg.norm(grad) * np.linalg.norm(grad_ref)))
    assert cos > 0.99
    assert np.linalg.norm(grad - grad_ref) <= 0.1 * np.linalg.norm(grad_ref)


def test_training_learns_the_level0_observable(dk):
    wl = W.get("mlmc16_256").with_(L_max=1)
    with dk.Context.from_workload(wl) as ctx:
        ctx.surrogate_init(3)
        r = ctx.surrogate_train(1 << 16, epochs=6, batch=512, lr=1e-3, seed=21)
        # variance of the target sqrt(N)(Y_0 - Ybar_0) = E[P_0] (about 0.26)
        s = ctx.run_level(0, 20000, seed=77)[0]
        var_t = s.pf1 / s.n
        assert r["val_mse"] < 0.2 * var_t, (r, var_t)
        corr = ctx.run_surrogate(0, 20000, seed=78)[0]
        v_corr = (corr.dp2 - corr.dp1 ** 2 / corr.n) / (corr.n - 1)
        v_p0 = (corr.pf2 - corr.pf1 ** 2 / corr.n) / (corr.n - 1)
        assert v_corr < 0.5 * v_p0, (v_corr, v_p0)
        print("surrogate train", r, "Var[P0 - S]/Var[P0] =", v_corr / v_p0)


@pytest.mark.parametrize("trained", [False, True])
def test_surrogate_estimate_is_unbiased(dk, trained):
    wl = W.get("mlmc16_256").with_(L_max=2)
    with dk.Context.from_workload(wl, pilot=400) as ctx:
        ctx.surrogate_init(5)
        if trained:
            ctx.surrogate_train(1 << 15, epochs=4, batch=512, lr=1e-3, seed=8)
        r_s, s_sur = ctx.estimate_surrogate(0.02, True, seed=31)
        r_p = ctx.estimate(0.02, True, seed=32)
    se = math.sqrt(r_s.variance + r_p.variance)
    assert abs(r_s.estimate - r_p.estimate) < 3.5 * se, (r_s.estimate, r_p.estimate, se)
    assert s_sur.n > 0 and r_s.M[0] > 0


@pytest.mark.parametrize("trained", [False, True])
def test_four_output_level_is_unbiased_for_every_quantity(dk, trained):
    """Four test functions with all products (10 quantities): the learned level
    plus its correction has the expectation of plain level 0 for each quantity
    (within 3.5 combined standard errors), trained or not; training lowers the
    correction's variance for the diagonal quantities."""
    import math
    wl = W.get("large32_1024").with_(L_max=1)
    n = 40000
    with dk.Context.from_workload(wl) as ctx:
        ctx.surrogate_init(11)
        if trained:
            r = ctx.surrogate_train(1 << 16, epochs=4, batch=512, lr=1e-3, seed=12)
            assert r["val_mse"] > 0
        s_sur = ctx.run_surrogate(-1, n, seed=13)
        s_cor = ctx.run_surrogate(0, n, seed=14)
        s_p0 = ctx.run_level(0, n, seed=15)
        assert ctx.n_quant == 10
        var = lambda q: (q.dp2 - q.dp1 ** 2 / q.n) / (q.n - 1)
        for q in range(ctx.n_quant):
            a, b, c = s_sur[q], s_cor[q], s_p0[q]
            assert a.n == b.n == c.n == n
            est = a.dp1 / n + b.dp1 / n
            ref = c.dp1 / n
            se = math.sqrt(var(a) / n + var(b) / n + var(c) / n)
            assert abs(est - ref) < 3.5 * se, (q, est, ref, se)
            if trained and q in (0, 4, 7, 9):   # diagonal quantities (j, j)
                assert var(b) < var(c), (q, var(b), var(c))


def test_theta_scheme_features_and_unbiasedness(dk):
    """The learned level on Crank--Nicolson levels: features with the theta
    factor (1 - b1 lam)/(1 + b0 lam) against the oracle, and the learned level
    plus its correction unbiased against plain level 0 (random network)."""
    wl = W.get("theta16_64").with_(L_max=1)
    n_s = 40000
    with dk.Context.from_workload(wl) as ctx:
        ctx.surrogate_init(3)
        info = ctx.level_info(0)
        X = ctx.surrogate_features(5, 4, seed=9, stream_tag=3)
        s_sur = ctx.run_surrogate(-1, n_s, seed=13)[0]
        s_cor = ctx.run_surrogate(0, n_s, seed=14)[0]
        s_p0 = ctx.run_level(0, n_s, seed=15)[0]
    n, M = info.n, info.M
    E, g = sg.modes(n), sg.heat_factors(n, info.tau / info.h ** 2, b0=wl.b0)
    sig = sg.feature_sigma(g, M)
    for i in range(4):
        Zs = [oracle.normals(9, 0, 3, 5 + i, m, n) for m in range(M)]
        np.testing.assert_allclose(X[i], sg.features(Zs, E, g) / sig, atol=2e-5, rtol=0)
    var = lambda q: (q.dp2 - q.dp1 ** 2 / q.n) / (q.n - 1)
    est = s_sur.dp1 / n_s + s_cor.dp1 / n_s
    se = math.sqrt(var(s_sur) / n_s + var(s_cor) / n_s + var(s_p0) / n_s)
    assert abs(est - s_p0.dp1 / n_s) < 3.5 * se
