"""Pins for the oracle's noise source (Definition 2.1: independent Brownian
increments per cell and component; the paper names no generator).

Philox4x32-10 is checked against the known-answer vectors published with the
Random123 library by the authors of Salmon et al. (SC'11); the normals are
checked for the counter layout and, statistically, for the standard normal
law that the increments Delta beta / sqrt(tau) must have.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


@pytest.mark.parametrize(
    "ctr,key,expect",
    [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ],
)
def test_philox_known_answers(ctr, key, expect):
    assert oracle.philox4x32_10(ctr, key) == expect


def _bm(a, b):
    u = (a + 1.0) / 2.0 ** 32
    th = 2.0 * math.pi * (b + 0.5) / 2.0 ** 32
    r = math.sqrt(-2.0 * math.log(u))
    return r * math.cos(th), r * math.sin(th)


@pytest.mark.parametrize("seed,level,stream,sample,m", [(0, 0, 0, 0, 0), (7, 3, 1, (5 << 32) + 11, 99)])
def test_counter_layout(seed, level, stream, sample, m):
    n = 8
    Z = oracle.normals(seed, level, stream, sample, m, n)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    tag = ((level + 1) & 0xFF) | ((stream & 0xFF) << 8) | (((sample >> 32) & 0xFFFF) << 16)
    for i1 in range(n):
        for i2 in range(n):
            p = (i1 * n + i2) // 2
            x = oracle.philox4x32_10([p, m, sample & 0xFFFFFFFF, tag], key)
            a, b = (x[0], x[1]) if (i1 * n + i2) % 2 == 0 else (x[2], x[3])
            z1, z2 = _bm(a, b)
            assert Z[i1, i2, 0] == pytest.approx(z1, abs=1e-14)
            assert Z[i1, i2, 1] == pytest.approx(z2, abs=1e-14)


def test_normals_are_standard_gaussian():
    Z = np.concatenate([oracle.normals(3, 2, 0, s, m, 64).reshape(-1) for s in range(4) for m in range(4)])
    assert Z.size == 64 * 64 * 2 * 16
    # Kolmogorov-Smirnov against the standard normal CDF, and the first four moments.
    assert stats.kstest(Z, "norm").pvalue > 1e-3
    se = 1.0 / math.sqrt(Z.size)
    assert abs(Z.mean()) < 5 * se
    assert abs(Z.var() - 1.0) < 5 * math.sqrt(2.0) * se
    assert abs(stats.kurtosis(Z, fisher=False) - 3.0) < 5 * math.sqrt(24.0) * se


def test_normals_independent_across_components_cells_steps_and_tags():
    a = oracle.normals(1, 0, 0, 0, 0, 64)
    b = oracle.normals(1, 0, 0, 0, 1, 64)        # next step
    c = oracle.normals(1, 1, 0, 0, 0, 64)        # next level tag
    d = oracle.normals(1, 0, 1, 0, 0, 64)        # plain-MC stream
    e = oracle.normals(1, 0, 0, 1, 0, 64)        # next sample
    f = oracle.normals(2, 0, 0, 0, 0, 64)        # next seed
    flat = [x.reshape(-1) for x in (a, b, c, d, e, f)]
    lim = 5.0 / math.sqrt(flat[0].size)
    for i in range(len(flat)):
        for j in range(i + 1, len(flat)):
            assert abs(np.corrcoef(flat[i], flat[j])[0, 1]) < lim
    assert abs(np.corrcoef(a[..., 0].reshape(-1), a[..., 1].reshape(-1))[0, 1]) < 2 * lim
    # neighbouring cells of one pair, and neighbouring pairs
    assert abs(np.corrcoef(a[:, 0::2, 0].reshape(-1), a[:, 1::2, 0].reshape(-1))[0, 1]) < 2 * lim
