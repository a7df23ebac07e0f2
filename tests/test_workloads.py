"""CPU checks of the synthetic workloads: every one describes a level
hierarchy the scheme accepts (Eq. cfl_preserved with its coupling's mesh
ratio, the stability bound of its time step), and its inputs have the shapes
of those grids.  The module holds inputs only; these checks use the oracle's
level table."""
import math

import numpy as np
import pytest

import oracle
from paper_2311_08872_gb300 import workloads as W


@pytest.mark.parametrize("name", sorted(W.WORKLOADS))
def test_workload_levels_and_inputs(name):
    wl = W.get(name)
    levels = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu, wl.M0, ratio=wl.ratio)
    mu = [lv.tau / lv.h ** 2 for lv in levels]
    assert all(abs(m - mu[0]) < 1e-9 * mu[0] for m in mu)           # tau / h^2 fixed over levels
    b1 = 1.0 - wl.b0
    if b1 > wl.b0:                                                    # stability of the noise-free step
        assert (b1 - wl.b0) * 2.0 * mu[0] <= 1.0 + 1e-12
    for l, lv in enumerate(levels):
        assert lv.n == wl.n(l) and lv.n % 2 == 0
        assert abs(lv.M * lv.tau - wl.T) < 1e-12 * wl.T
        if l > 0:
            assert lv.M % (wl.ratio ** 2) == 0 and lv.n % wl.ratio == 0
        rho0 = wl.rho0(l)
        assert rho0.shape == (lv.n, lv.n) and np.all(np.isfinite(rho0))
        for p in wl.phi(l):
            assert p.shape == (lv.n, lv.n) and np.all(np.isfinite(p))
    if wl.coupling == 1:
        assert wl.n0 == 6 and wl.L_max <= 3      # 6^2 .. 162^2
    if wl.b0 > 0:
        assert wl.n(wl.L_max) <= 128      # the theta kernels: one CTA up to 64^2, 4-CTA clusters at 128^2


def test_cell_centred_workload_is_the_shifted_grid():
    """The symmetric-coupling workload samples the same functions half a cell
    further (Remark avoid_right_bias)."""
    a, b = W.get("mlmc16_256"), W.get("mlmc16_256_sym")
    n = a.n(0)
    x1, x2 = W.grid_coords(n, 1.0, 0.5)
    np.testing.assert_allclose(b.rho0(0), W.rho0_sinsin(x1, x2, 1.0), rtol=0, atol=1e-15)
    assert not np.allclose(a.rho0(0), b.rho0(0))
    assert math.isclose(b.offset, 0.5)
