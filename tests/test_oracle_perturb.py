"""Pins of the oracle's perturbation hook (oracle_sample_perturbed).

On ill-conditioned low-density levels the GPU parity bar is set by the
oracle's own response to rounding-sized perturbations, so the hook itself must
be right: with amp = 0 it is the plain oracle sample bit for bit; every
perturbation conserves mass; each edge transfer is uniform on [-amp/2, amp/2)
and enters in divergence form with the stated orientation; and on the
noise-free linear scheme (Eq. FullyDiscreteDK with N^-1/2 = 0, the heat
scheme of Section 7.2) the variance of the change of (rho^M, cos 2 pi x1)_h
has a closed form in amp, so an amplitude off by any factor fails.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_08872_gb300 import workloads as W


def _level(wl, level, coupled, **kw):
    wl = wl.with_(**kw) if kw else wl
    levels = oracle.level_table(wl.length, wl.n0, wl.L_max, wl.T, wl.mu, wl.M0)
    return oracle.level_inputs(wl.length, levels, wl.N, wl.rho0_all(), wl.phi_all(), level, coupled), levels


@pytest.mark.parametrize("name,level", [("mlmc16_256", 1), ("lowdens32_512", 1)])
def test_zero_amplitude_is_the_plain_sample(name, level):
    ol, _ = _level(W.get(name), level, True)
    for i in (0, 7):
        a = ol.sample(3, i, True)
        b = ol.sample_perturbed(3, i, True, 0.0, 99)
        assert np.array_equal(a["Y_f"], b["Y_f"]) and np.array_equal(a["Y_c"], b["Y_c"])
        assert a["mass_f"] == b["mass_f"] and a["mass_c"] == b["mass_c"]


def test_perturbation_conserves_mass():
    rng = np.random.default_rng(5)
    for n in (8, 33, 64):
        rho = rng.uniform(0.0, 2.0, (n, n))
        out, _ = oracle.perturb_field(n, 1e-3, 17, rho)
        assert abs(out.sum() - rho.sum()) <= 1e-14 * rho.sum()
        assert np.any(out != rho)
    # along whole coupled paths, with noise (mass to rounding of the FP64 sums)
    ol, _ = _level(W.get("lowdens32_512"), 1, True)
    base = ol.sample(2, 0, True)
    p = ol.sample_perturbed(2, 0, True, 2.0 ** -20, 1)
    assert abs(p["mass_f"] - base["mass_f"]) <= 1e-13
    assert abs(p["mass_c"] - base["mass_c"]) <= 1e-13


def test_transfer_law_and_orientation():
    n, amp = 64, 0.25
    rho = np.zeros((n, n))
    out, tr = oracle.perturb_field(n, amp, 2024, rho)
    e1, e2 = tr[..., 0], tr[..., 1]
    # each cell gains its own two edge transfers and loses those of the edges
    # it closes from above (component 1) and from the left (component 2)
    div = e1 + e2 - np.roll(e1, 1, axis=0) - np.roll(e2, 1, axis=1)
    np.testing.assert_allclose(out, div, rtol=0, atol=1e-15)
    e = tr.reshape(-1)
    assert np.all(e >= -amp / 2) and np.all(e < amp / 2)
    # uniform on [-amp/2, amp/2): mean 0, variance amp^2/12, flat histogram
    k = e.size
    assert abs(e.mean()) < 4 * amp / math.sqrt(12 * k)
    var = e.var()
    assert abs(var / (amp * amp / 12) - 1) < 4 * math.sqrt(0.8 / k)     # Var of U^2 is (4/5)(amp^2/12)^2
    hist, _ = np.histogram(e, bins=16, range=(-amp / 2, amp / 2))
    expect = k / 16
    chi2 = float(np.sum((hist - expect) ** 2 / expect))
    assert chi2 < 45.0                                                  # 15 dof: p ~ 1e-4
    # consecutive draws uncorrelated
    assert abs(np.corrcoef(e[:-1], e[1:])[0, 1]) < 4 / math.sqrt(k)
    # a different stream gives different transfers, the same stream the same
    _, tr2 = oracle.perturb_field(n, amp, 2025, rho)
    _, tr3 = oracle.perturb_field(n, amp, 2024, rho)
    assert not np.array_equal(tr, tr2) and np.array_equal(tr, tr3)


def test_response_of_the_linear_scheme_has_the_closed_form_variance():
    """N^-1/2 = 0: the scheme is the linear heat scheme, the perturbation after
    fine step m reaches T multiplied by g^(M-1-m) on the mode cos(2 pi x1), and
    an edge transfer e along component 1 changes (rho, phi)_h by
    h^2 e (phi(x) - phi(x + h e1)) (component 2 leaves this phi unchanged).
    Summing the independent uniform transfers, for h = 1/n,
        Var[dY] = (amp^2 / 6) h^2 sin^2(pi h) (1 - g^(2M)) / (1 - g^2),
    g = 1 - 2 (tau/h^2) sin^2(pi h)."""
    wl = W.get("mlmc16_256")
    ol, levels = _level(wl, 0, False, N=0.0)
    lv = levels[0]
    amp = 1e-6
    base = ol.sample(1, 0, False)["Y_f"][0]
    d = np.array([ol.sample_perturbed(1, 0, False, amp, 1000 + r)["Y_f"][0] - base for r in range(400)])
    h, n = lv.h, lv.n
    g = 1.0 - 2.0 * (lv.tau / (h * h)) * math.sin(math.pi * h) ** 2
    expect = amp * amp / 6.0 * h * h * math.sin(math.pi * h) ** 2 * (1 - g ** (2 * lv.M)) / (1 - g * g)
    assert abs(d.mean()) < 4 * math.sqrt(expect / d.size)
    ratio = float(np.mean(d * d)) / expect
    # 400 draws of a (nearly) Gaussian dY: the mean square is within ~4 x sqrt(2/400) = 28%
    assert 0.72 < ratio < 1.28, ratio
    # linear in amp
    d2 = np.array([ol.sample_perturbed(1, 0, False, 2 * amp, 1000 + r)["Y_f"][0] - base for r in range(8)])
    np.testing.assert_allclose(d2, 2 * d[:8], rtol=1e-6)
