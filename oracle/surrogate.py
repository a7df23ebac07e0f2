"""FP64 oracle for the learned level below level 0 (not in the paper).

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``).

* ``modes(n, count)``: the lowest real orthonormal Fourier modes of an n x n
  grid (orthonormal for the plain sum over grid points), excluding the
  constant: wave vectors k with k1 > 0, or k1 = 0 and k2 > 0, ordered by
  |k|^2 then (k1, k2); each contributes a cosine and a sine mode.
* ``features(Z, g)``: heat-weighted projections F_(j, r) = sum_m g_j^(M-1-m)
  <Z^m_(., r), e_j> of the level-0 normals on the modes e_j (component r of
  the noise), with g_j the per-step factor of the noise-free scheme on mode j
  (the discrete heat symbol of Section 7.2's operators).  With i.i.d. N(0,1)
  normals and orthonormal modes they are independent N(0, sum_i g_j^(2i)).
* ``mlp_*``: a plain FP64 4-layer ReLU perceptron 64-256-256-256-K, one
  output per test function (forward, backward, squared-error loss summed over
  the outputs) for checking the GPU kernels.

Pins (tests/test_oracle_surrogate.py): the modes' orthonormality, the
features' exact Gaussian law, the MLP gradient against central finite
differences.  Parity unpinned: the values of a trained network (the paper
has no learned level, so nothing fixes them beyond these properties).
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np


def mode_vectors(n: int, count: int) -> List[Tuple[int, int]]:
    ks = []
    half = n // 2
    for k1 in range(0, half + 1):
        for k2 in range(-half + 1, half + 1):
            if k1 == 0 and k2 <= 0:
                continue
            if 2 * k1 == n or 2 * abs(k2) == n:
                continue   # Nyquist lines: no sine partner
            ks.append((k1, k2))
    ks.sort(key=lambda k: (k[0] * k[0] + k[1] * k[1], k[0], k[1]))
    return ks[: (count + 1) // 2]


def modes(n: int, count: int = 32) -> np.ndarray:
    """E of shape (count, n, n): cos/sin pairs, orthonormal for the plain sum."""
    i1, i2 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    out = []
    for k1, k2 in mode_vectors(n, count):
        ang = 2 * math.pi * (k1 * i1 + k2 * i2) / n
        out.append(math.sqrt(2.0 / (n * n)) * np.cos(ang))
        out.append(math.sqrt(2.0 / (n * n)) * np.sin(ang))
    return np.array(out[:count])


def heat_factors(n: int, mu: float, count: int = 32, b0: float = 0.0) -> np.ndarray:
    """Per-step factor of each mode under the noise-free scheme: with
    lam = 2 mu (sin^2(pi k1/n) + sin^2(pi k2/n)), (1 - b1 lam)/(1 + b0 lam) for
    the weights (b0, b1 = 1 - b0) of Eq. (FullyDiscreteDK) (1 - lam explicit)."""
    g = []
    for k1, k2 in mode_vectors(n, count):
        lam = 2.0 * mu * (math.sin(math.pi * k1 / n) ** 2 + math.sin(math.pi * k2 / n) ** 2)
        gk = (1.0 - (1.0 - b0) * lam) / (1.0 + b0 * lam)
        g += [gk, gk]
    return np.array(g[:count])


def feature_sigma(g: np.ndarray, M: int) -> np.ndarray:
    """Standard deviation of each feature: sqrt(sum_{i<M} g^(2i)), per (mode, component)."""
    s = np.sqrt(np.array([np.sum(gk ** (2 * np.arange(M))) for gk in g]))
    return np.repeat(s, 2)


def features(Zs: List[np.ndarray], E: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Zs: the M arrays of normals (n, n, 2) of one sample, in step order.
    Returns the 2*count features ordered (mode j, component r) -> 2 j + r."""
    M = len(Zs)
    F = np.zeros((E.shape[0], 2))
    for m, Z in enumerate(Zs):
        w = g ** (M - 1 - m)
        for r in range(2):
            F[:, r] += w * np.tensordot(E, Z[..., r], axes=([1, 2], [0, 1]))
    return F.reshape(-1)


# ------------------------------------------------------------------- MLP
LAYERS = (64, 256, 256, 256, 1)


def layers(outputs: int = 1):
    """Widths of the 4-layer perceptron with `outputs` outputs (one per test function)."""
    return LAYERS[:-1] + (outputs,)


def mlp_param_count(outputs: int = 1) -> int:
    w = layers(outputs)
    return sum(w[i] * w[i + 1] + w[i + 1] for i in range(len(w) - 1))


def mlp_unpack(theta: np.ndarray, outputs: int = 1):
    """Flat parameter vector -> [(W [out, in], b [out])], layer by layer (W then b)."""
    w = layers(outputs)
    out, off = [], 0
    for i in range(len(w) - 1):
        a, b = w[i], w[i + 1]
        W = theta[off: off + a * b].reshape(b, a)
        off += a * b
        bias = theta[off: off + b]
        off += b
        out.append((W, bias))
    return out


def mlp_forward(theta: np.ndarray, X: np.ndarray, outputs: int = 1):
    """Outputs y of shape (B,) for one output, (B, outputs) otherwise, and the activations."""
    acts = [X]
    h = X
    ls = mlp_unpack(theta, outputs)
    for i, (W, b) in enumerate(ls):
        z = h @ W.T + b
        h = np.maximum(z, 0.0) if i < len(ls) - 1 else z
        acts.append(h)
    return (h[:, 0] if outputs == 1 else h), acts


def mlp_loss_grad(theta: np.ndarray, X: np.ndarray, T: np.ndarray):
    """Squared error summed over the outputs, averaged over the batch (the mean
    squared error for one output), and its gradient (flat, layout of theta).
    T: (B,) for one output, (B, outputs) otherwise."""
    T2 = T[:, None] if T.ndim == 1 else T
    outputs = T2.shape[1]
    y, acts = mlp_forward(theta, X, outputs)
    y2 = y[:, None] if outputs == 1 else y
    B = X.shape[0]
    loss = float(np.sum((y2 - T2) ** 2) / B)
    d = (2.0 / B) * (y2 - T2)
    ls = mlp_unpack(theta, outputs)
    grads = []
    for i in range(len(ls) - 1, -1, -1):
        W, b = ls[i]
        h_in = acts[i]
        gW = d.T @ h_in
        gb = d.sum(axis=0)
        grads.append((gW, gb))
        if i > 0:
            d = (d @ W) * (acts[i] > 0)
    flat = []
    for gW, gb in reversed(grads):
        flat += [gW.reshape(-1), gb]
    return loss, np.concatenate(flat)
