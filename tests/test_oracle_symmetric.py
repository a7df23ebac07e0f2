"""Pins for the symmetric variant of the NN coupling (Remark avoid_right_bias):
the same index coupling (coarse cell I takes the fine block {2I, 2I+1}^2) on
cell-centred grids, where each coarse point is the centre of its block.

* Mirror symmetry (exact, chosen noise): reflecting the torus in x1 maps the
  cell-centred fine and coarse grids, and each coupled block, onto
  themselves.  Driving a coupled pair with the mirrored fine noise (component
  1 changes sign) therefore mirrors both paths, and for mirror-even rho0 and
  phi leaves Y_f and Y_c unchanged to rounding.  On the vertex grid of the
  Right-Most coupling the fine path is still mirrored but the blocks are not
  (the mirror of {2I, 2I+1} is {2J-1, 2J}), so Y_c changes: the test tells
  the two couplings apart.
* The martingale-lemma closed form of E[P] holds on the cell-centred grid
  (its derivation only uses sums of sin/cos over a full period).
* The coarse member of a pair has the law of a stand-alone coarser path
  (Remark distribution_W_ell) on the cell-centred grids too.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_08872_gb300 import workloads as W

K_SE = 3.5


def _even_rho0(n, offset):
    x1, x2 = W.grid_coords(n, 1.0, offset)
    return 1.0 + 0.5 * np.cos(2 * math.pi * x1) * np.cos(2 * math.pi * x2)


def _cos1(n, offset):
    x1, _ = W.grid_coords(n, 1.0, offset)
    return np.cos(2 * math.pi * x1)


def _mirror_noise(Z, offset):
    """Fine normals of the mirrored path: x1 -> -x1, so the cell index maps
    i1 -> n-1-i1 on the cell-centred grid and i1 -> -i1 mod n on the vertex
    grid, and component 1 (along x1) changes sign."""
    n = Z.shape[1]
    idx = (n - 1 - np.arange(n)) if offset == 0.5 else (-np.arange(n)) % n
    Zm = Z[:, idx, :, :].copy()
    Zm[..., 0] *= -1.0
    return Zm


@pytest.mark.parametrize("offset", [0.5, 0.0])
def test_mirror_symmetry_of_the_coupling(offset):
    levels = oracle.level_table(1.0, 8, 1, 0.004, 0.1)
    lv = levels[1]
    n, nc = lv.n, lv.n // 2
    ol = oracle.OracleLevel(lv, 400.0, _even_rho0(n, offset), [_cos1(n, offset)],
                            _even_rho0(nc, offset), [_cos1(nc, offset)])
    rng = np.random.default_rng(11)
    Z = rng.standard_normal((lv.M, n, n, 2))
    a = ol.sample_given(Z, coupled=True, fields=True)
    b = ol.sample_given(_mirror_noise(Z, offset), coupled=True, fields=True)
    scale = abs(a["Y_f"][0]) + 1e-3
    # the fine path is mirrored on either grid
    assert abs(a["Y_f"][0] - b["Y_f"][0]) < 1e-12 * scale
    idx = (n - 1 - np.arange(n)) if offset == 0.5 else (-np.arange(n)) % n
    np.testing.assert_allclose(b["rho_f"], a["rho_f"][idx, :], rtol=0, atol=1e-13)
    dc = abs(a["Y_c"][0] - b["Y_c"][0])
    if offset == 0.5:
        cidx = nc - 1 - np.arange(nc)
        np.testing.assert_allclose(b["rho_c"], a["rho_c"][cidx, :], rtol=0, atol=1e-13)
        assert dc < 1e-12 * scale
    else:
        assert dc > 1e-6 * scale, dc


def test_closed_form_mean_of_P_on_cell_centred_grid():
    N = 1e8
    lv = oracle.level_table(1.0, 16, 0, 0.02, 0.1)[0]
    wl = W.get("mlmc16_256_sym")
    rho0, phi = wl.rho0(0), wl.phi(0)
    ol = oracle.OracleLevel(lv, N, rho0, phi)
    r = oracle.run_samples(ol, seed=17, ids=range(2500), coupled=False, stream=1)
    Ybar = oracle.inner_h(oracle.mean_field(16, lv.h, lv.tau, lv.M, rho0), phi[0], lv.h)
    P = oracle.observable_P(N, r["Y_f"], [Ybar])[:, 0]
    se = P.std(ddof=1) / math.sqrt(P.size)
    expect = oracle.closed_form_EP_cos1(1.0, 16, lv.tau, lv.M)
    assert abs(P.mean() - expect) < K_SE * se
    assert se / expect < 0.05


def test_coarse_member_has_standalone_law_on_cell_centred_grids():
    wl = W.get("mlmc16_256_sym").with_(n0=8, L_max=1, N=2e3)
    levels = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu)
    rho0, phi = wl.rho0_all(), wl.phi_all()
    pair = oracle.level_inputs(wl.length, levels, wl.N, rho0, phi, 1, True)
    single = oracle.level_inputs(wl.length, levels, wl.N, rho0, phi, 0, False)
    rp = oracle.run_samples(pair, seed=5, ids=range(1500), coupled=True)
    rs = oracle.run_samples(single, seed=6, ids=range(1500), coupled=False)
    lv0 = levels[0]
    Ybar = oracle.inner_h(oracle.mean_field(lv0.n, lv0.h, lv0.tau, lv0.M, rho0[0]), phi[0][0], lv0.h)
    Pc = oracle.observable_P(wl.N, rp["Y_c"], [Ybar])[:, 0]
    Ps = oracle.observable_P(wl.N, rs["Y_f"], [Ybar])[:, 0]
    se = math.sqrt(Pc.var(ddof=1) / Pc.size + Ps.var(ddof=1) / Ps.size)
    assert abs(Pc.mean() - Ps.mean()) < K_SE * se
    vc, vs = Pc.var(ddof=1), Ps.var(ddof=1)
    se_v = math.sqrt(2.0 / (Pc.size - 1)) * max(vc, vs) * 2.0
    assert abs(vc - vs) < K_SE * se_v
