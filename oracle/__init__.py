"""FP64 oracle for the coupled Dean--Kawasaki MLMC hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) may import
this package.  It shares no code with the CUDA path and never imports the
product package; inputs (rho0 and phi on the grids, seeds) are passed in as
arrays.

Contents, each following the paper (Cornalba & Fischer, arXiv 2311.08872):
  * ``liboracle_dk.so`` (dk_oracle.c): Philox4x32-10, Box--Muller normals, one
    step of Eq. (FullyDiscreteDK) with b0=0, b1=1 (Section 7.2) and with
    general weights b0 + b1 = 1 (theta-scheme, exact periodic solve), the
    Right-Most NN coupled pair of Section 3.2, the discrete mean field.
  * ``level_table``: the CFL-linked level hierarchy of Eq. (cfl_preserved)
    with h_{l-1} = 2 h_l, tau_{l-1} = 4 tau_l (Section 7.2).
  * ``observable_P``: P_l of Eq. (eqn_MLMCLevels) with psi(x) = x^2.
  * ``mlmc_*``: the estimator of Eq. (MLMCEstimator), the sample allocation of
    Eq. (opt_M_ell), the stopping test of Eq. (convergence_criterion) and
    Algorithm 1 (Section 7.1).
  * closed forms used as pins: the discrete heat symbol, and E[P] from the
    discrete martingale lemma (Appendix C, Lemma lem_Discrete_Martingale).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

_LIB = None

_dp = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)


class _OracleLevelC(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("h", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("M", ctypes.c_int64),
        ("level", ctypes.c_int),
        ("inv_sqrt_N", ctypes.c_double),
        ("rho0_f", _dp),
        ("rho0_c", _dp),
        ("n_obs", ctypes.c_int),
        ("phi_f", _dp),
        ("phi_c", _dp),
        ("b0", ctypes.c_double),
        ("coupling", ctypes.c_int),
    ]


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.oracle_normals.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.c_int64, ctypes.c_int, _dp]
        L.oracle_dk_step.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     _dp, _dp, _dp]
        L.oracle_sample.argtypes = [ctypes.POINTER(_OracleLevelC), ctypes.c_uint64, ctypes.c_int,
                                    ctypes.c_uint64, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
        L.oracle_sample.restype = ctypes.c_int
        L.oracle_sample_perturbed.argtypes = [ctypes.POINTER(_OracleLevelC), ctypes.c_uint64, ctypes.c_int,
                                              ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                              _dp, _dp, _dp, _dp]
        L.oracle_sample_perturbed.restype = ctypes.c_int
        L.oracle_perturb_field.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint64, _dp, _dp]
        L.oracle_sample_given.argtypes = [ctypes.POINTER(_OracleLevelC), _dp, ctypes.c_int,
                                          _dp, _dp, _dp, _dp, _dp, _dp]
        L.oracle_sample_given.restype = ctypes.c_int
        L.oracle_mean_field.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                        _dp, _dp]
        L.oracle_theta_step.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, _dp, _dp, _dp]
        L.oracle_helmholtz_solve.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
        L.oracle_fourier_restrict.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
        L.oracle_mean_field_theta.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                              ctypes.c_double, _dp, _dp]
        _LIB = L
    return _LIB


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


# ------------------------------------------------------------------- noise
def philox4x32_10(ctr: Sequence[int], key: Sequence[int]) -> List[int]:
    """Philox4x32-10 of Salmon et al. (SC'11) on one 128-bit counter."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return list(o)


def normals(seed: int, level: int, stream: int, sample: int, m: int, n: int) -> np.ndarray:
    """Z of shape (n, n, 2): the standard normals driving fine step m."""
    Z = np.empty((n, n, 2), dtype=np.float64)
    lib().oracle_normals(seed, level, stream, sample, m, n, _ptr(Z))
    return Z


def dk_step(n: int, h: float, tau: float, inv_sqrt_N: float, rho: np.ndarray,
            dbeta: Optional[np.ndarray]) -> np.ndarray:
    """One explicit Euler--Maruyama step of Eq. (FullyDiscreteDK)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.empty_like(rho)
    db = None if dbeta is None else np.ascontiguousarray(dbeta, dtype=np.float64)
    lib().oracle_dk_step(n, h, tau, inv_sqrt_N, _ptr(rho), _ptr(db), _ptr(out))
    return out


def theta_step(n: int, h: float, tau: float, inv_sqrt_N: float, b0: float, rho: np.ndarray,
               dbeta: Optional[np.ndarray]) -> np.ndarray:
    """One step of Eq. (FullyDiscreteDK) with weights (b0, 1 - b0)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.empty_like(rho)
    db = None if dbeta is None else np.ascontiguousarray(dbeta, dtype=np.float64)
    lib().oracle_theta_step(n, h, tau, inv_sqrt_N, b0, _ptr(rho), _ptr(db), _ptr(out))
    return out


def helmholtz_solve(n: int, c: float, rhs: np.ndarray) -> np.ndarray:
    """(I + c L)^{-1} rhs on the periodic grid, L = -h^2 Delta_h (5-point)."""
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    out = np.empty_like(rhs)
    lib().oracle_helmholtz_solve(n, c, _ptr(rhs), _ptr(out))
    return out


def fourier_restrict(n: int, nc: int, fine: np.ndarray) -> np.ndarray:
    """The coarse field of the Fourier coupling (Section 3.1) carrying the modes
    of the fine field that the nc x nc grid resolves (see oracle_fourier_restrict)."""
    fine = np.ascontiguousarray(fine, dtype=np.float64).reshape(n, n)
    out = np.empty((nc, nc))
    lib().oracle_fourier_restrict(n, nc, _ptr(fine), _ptr(out))
    return out


def mean_field(n: int, h: float, tau: float, M: int, rho0: np.ndarray, b0: float = 0.0) -> np.ndarray:
    """The discrete mean field rho-bar: the noise-free scheme iterated M times
    (weights (b0, 1 - b0) of Eq. FullyDiscreteDK)."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    out = np.empty_like(rho0)
    if b0 == 0.0:
        lib().oracle_mean_field(n, h, tau, M, _ptr(rho0), _ptr(out))
    else:
        lib().oracle_mean_field_theta(n, h, tau, M, b0, _ptr(rho0), _ptr(out))
    return out


def inner_h(f: np.ndarray, g: np.ndarray, h: float) -> float:
    """(f, g)_h = h^d sum_x f(x) g(x) (Section 2)."""
    return float(h * h * np.sum(f * g))


# ----------------------------------------------------------- level table
@dataclass
class Level:
    level: int
    n: int
    h: float
    tau: float
    M: int


def level_table(length: float, n0: int, L_max: int, T: float, mu: float, M0: int = 0, ratio: int = 2) -> List[Level]:
    """Levels with tau_l / h_l^2 fixed (Eq. cfl_preserved), h_{l-1} = r h_l and
    tau_{l-1} = r^2 tau_l: r = 2 for the NN coupling (Section 7.2), r = 3 for
    the Fourier coupling (Section 3.1).  T / tau_0 must be an integer; where the
    nominal mu does not give one, M_0 = ceil(T / (mu h_0^2)) and tau_0 = T / M_0,
    so the effective ratio is at most mu and the same on every level."""
    h0 = length / n0
    if M0 <= 0:
        x = T / (mu * h0 * h0)
        M0 = int(math.ceil(x - 1e-9 * x))
    tau0 = T / M0
    k = ratio * ratio
    return [Level(l, n0 * ratio ** l, h0 / ratio ** l, tau0 / (k ** l), M0 * (k ** l)) for l in range(L_max + 1)]


# ---------------------------------------------------------------- samples
class OracleLevel:
    """Inputs of one level for the C oracle (arrays kept alive here)."""

    def __init__(self, lv: Level, N: float, rho0_f: np.ndarray, phi_f: Sequence[np.ndarray],
                 rho0_c: Optional[np.ndarray] = None, phi_c: Optional[Sequence[np.ndarray]] = None,
                 b0: float = 0.0, coupling: int = 0):
        self.lv = lv
        self.N = N
        self.b0 = float(b0)
        self.coupling = int(coupling)
        self.n_obs = len(phi_f)
        self.rho0_f = np.ascontiguousarray(rho0_f, dtype=np.float64).reshape(-1)
        self.phi_f = np.ascontiguousarray(np.stack(phi_f), dtype=np.float64)
        self.rho0_c = None if rho0_c is None else np.ascontiguousarray(rho0_c, dtype=np.float64).reshape(-1)
        self.phi_c = None if phi_c is None else np.ascontiguousarray(np.stack(phi_c), dtype=np.float64)
        self.c = _OracleLevelC(lv.n, lv.h, lv.tau, lv.M, lv.level,
                               0.0 if not N else 1.0 / math.sqrt(N),
                               _ptr(self.rho0_f), _ptr(self.rho0_c), self.n_obs,
                               _ptr(self.phi_f), _ptr(self.phi_c), self.b0, self.coupling)

    def sample(self, seed: int, sample: int, coupled: bool, stream: int = 0, fields: bool = False):
        n = self.lv.n
        Yf = np.zeros(self.n_obs)
        Yc = np.zeros(self.n_obs)
        mf = ctypes.c_double(0.0)
        mc = ctypes.c_double(0.0)
        rf = np.empty(n * n) if fields else None
        nc = n // (3 if self.coupling == 1 else 2)
        rc = np.empty(nc * nc) if (fields and coupled) else None
        rc_ = lib().oracle_sample(ctypes.byref(self.c), seed, stream, sample, int(coupled),
                                  _ptr(Yf), _ptr(Yc), ctypes.byref(mf), ctypes.byref(mc),
                                  _ptr(rf), _ptr(rc))
        if rc_ != 0:
            raise ValueError(f"oracle_sample failed ({rc_})")
        out = dict(Y_f=Yf, Y_c=Yc if coupled else None, mass_f=mf.value,
                   mass_c=mc.value if coupled else None)
        if fields:
            out["rho_f"] = rf.reshape(n, n)
            if coupled:
                out["rho_c"] = rc.reshape(nc, nc)
        return out


    def sample_given(self, Z: np.ndarray, coupled: bool, fields: bool = False):
        """The sample driven by the caller's fine normals Z of shape (M, n, n, 2)
        (see oracle_sample_given)."""
        n, M = self.lv.n, self.lv.M
        Z = np.ascontiguousarray(Z, dtype=np.float64)
        if Z.shape != (M, n, n, 2):
            raise ValueError(f"normals must have shape {(M, n, n, 2)}")
        Yf = np.zeros(self.n_obs)
        Yc = np.zeros(self.n_obs)
        mf = ctypes.c_double(0.0)
        mc = ctypes.c_double(0.0)
        rf = np.empty(n * n) if fields else None
        nc = n // (3 if self.coupling == 1 else 2)
        rc = np.empty(nc * nc) if (fields and coupled) else None
        rc_ = lib().oracle_sample_given(ctypes.byref(self.c), _ptr(Z), int(coupled), _ptr(Yf), _ptr(Yc),
                                        ctypes.byref(mf), ctypes.byref(mc), _ptr(rf), _ptr(rc))
        if rc_ != 0:
            raise ValueError(f"oracle_sample_given failed ({rc_})")
        out = dict(Y_f=Yf, Y_c=Yc if coupled else None, mass_f=mf.value, mass_c=mc.value if coupled else None)
        if fields:
            out["rho_f"] = rf.reshape(n, n)
            if coupled:
                out["rho_c"] = rc.reshape(nc, nc)
        return out

    def sample_perturbed(self, seed: int, sample: int, coupled: bool, amp: float, perturb_seed: int,
                         stream: int = 0):
        """The same sample with mass-conserving random edge transfers of size
        amp after every step (see oracle_sample_perturbed)."""
        Yf = np.zeros(self.n_obs)
        Yc = np.zeros(self.n_obs)
        mf = ctypes.c_double(0.0)
        mc = ctypes.c_double(0.0)
        rc_ = lib().oracle_sample_perturbed(ctypes.byref(self.c), seed, stream, sample, int(coupled), amp,
                                            perturb_seed, _ptr(Yf), _ptr(Yc), ctypes.byref(mf), ctypes.byref(mc))
        if rc_ != 0:
            raise ValueError(f"oracle_sample_perturbed failed ({rc_})")
        return dict(Y_f=Yf, Y_c=Yc if coupled else None, mass_f=mf.value, mass_c=mc.value if coupled else None)


def perturb_field(n: int, amp: float, perturb_seed: int, rho: np.ndarray):
    """The perturbation oracle_sample_perturbed applies after a step, on a copy
    of the n x n field rho: returns (perturbed field, transfers [n, n, 2])."""
    out = np.ascontiguousarray(rho, dtype=np.float64).reshape(n, n).copy()
    tr = np.empty((n, n, 2))
    lib().oracle_perturb_field(n, amp, perturb_seed, _ptr(out), _ptr(tr))
    return out, tr


def level_inputs(length: float, levels: List[Level], N: float, rho0: List[np.ndarray],
                 phi: List[List[np.ndarray]], level: int, coupled: bool, b0: float = 0.0,
                 coupling: int = 0) -> OracleLevel:
    lv = levels[level]
    if coupled and level > 0:
        return OracleLevel(lv, N, rho0[level], phi[level], rho0[level - 1], phi[level - 1], b0=b0, coupling=coupling)
    return OracleLevel(lv, N, rho0[level], phi[level], b0=b0, coupling=coupling)


def _run_chunk(args):
    (lv, N, rho0_f, phi_f, rho0_c, phi_c, seed, ids, coupled, stream, b0, coupling) = args
    ol = OracleLevel(lv, N, rho0_f, phi_f, rho0_c, phi_c, b0=b0, coupling=coupling)
    res = [ol.sample(seed, int(i), coupled, stream) for i in ids]
    return res


def run_samples(ol: OracleLevel, seed: int, ids: Sequence[int], coupled: bool, stream: int = 0,
                processes: int = 1):
    """Per-sample outputs for the given sample ids, as arrays.

    With processes > 1 a ``spawn`` pool runs disjoint chunks, each process
    single-threaded."""
    ids = list(ids)
    if processes <= 1 or len(ids) <= 1:
        res = [ol.sample(seed, i, coupled, stream) for i in ids]
    else:
        import multiprocessing as mp
        chunks = [ids[i::processes] for i in range(processes)]
        args = [(ol.lv, ol.N, ol.rho0_f, list(ol.phi_f), ol.rho0_c,
                 None if ol.phi_c is None else list(ol.phi_c), seed, c, coupled, stream, ol.b0, ol.coupling)
                for c in chunks if c]
        with mp.get_context("spawn").Pool(len(args)) as pool:
            parts = pool.map(_run_chunk, args)
        by_id = {}
        for c, part in zip([c for c in chunks if c], parts):
            for i, r in zip(c, part):
                by_id[i] = r
        res = [by_id[i] for i in ids]
    Yf = np.array([r["Y_f"] for r in res])
    Yc = np.array([r["Y_c"] for r in res]) if coupled else None
    mf = np.array([r["mass_f"] for r in res])
    mc = np.array([r["mass_c"] for r in res]) if coupled else None
    return dict(Y_f=Yf, Y_c=Yc, mass_f=mf, mass_c=mc)


# ------------------------------------------------------------ observables
def observable_P(N: float, Y: np.ndarray, Ybar: np.ndarray, products: bool = False) -> np.ndarray:
    """P = psi(N^{1/2} (Y - Ybar)) with psi(x) = x^2 (Eq. eqn_MLMCLevels).

    With ``products`` the quantities are N (Y_j - Ybar_j)(Y_k - Ybar_k) for
    all j <= k (the squares included), in row-major order of (j, k)."""
    D = np.atleast_2d(Y) - np.asarray(Ybar)[None, :]
    if not products:
        return N * D * D
    cols = []
    K = D.shape[1]
    for j in range(K):
        for k in range(j, K):
            cols.append(N * D[:, j] * D[:, k])
    return np.stack(cols, axis=1)


# ------------------------------------------------------------ MLMC driver
def mlmc_optimal_samples(V: Sequence[float], C: Sequence[float], eps: float) -> List[int]:
    """Eq. (opt_M_ell): M_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_j sqrt(V_j C_j))."""
    total = sum(math.sqrt(v * c) for v, c in zip(V, C))
    return [int(math.ceil(2.0 / (eps * eps) * math.sqrt(v / c) * total)) for v, c in zip(V, C)]


def mlmc_converged(E: Sequence[float], eps: float, alpha: float = 2.0, ratio: float = 2.0) -> bool:
    """Eq. (convergence_criterion): stop on level L if
    max_{t in {0,1,2}} 2^{-t alpha} |E[P_{L-t} - P_{L-t-1}]| / (2^alpha - 1) < eps / sqrt 2,
    with P_{-1} = 0 (levels below 0 are skipped).  The 2 is the mesh ratio of
    the NN hierarchy; `ratio` = 3 for the Fourier coupling's levels."""
    L = len(E) - 1
    worst = 0.0
    for t in range(3):
        if L - t < 0:
            break
        worst = max(worst, ratio ** (-t * alpha) * abs(E[L - t]))
    return worst / (ratio ** alpha - 1.0) < eps / math.sqrt(2.0)


def mlmc_estimator(sums_dp: Sequence[float], counts: Sequence[int]) -> float:
    """Eq. (MLMCEstimator): sum over levels of the sample mean of P_l - P_{l-1}."""
    return float(sum(s / m for s, m in zip(sums_dp, counts)))


# ----------------------------------------------------------- closed forms
def heat_symbol(k: Sequence[int], n: int, mu: float, b0: float = 0.0) -> float:
    """Per-step factor of the noise-free scheme on the discrete Fourier mode
    exp(2 pi i k.x / L): with lam = 2 (tau/h^2) (sin^2(pi k1/n) + sin^2(pi k2/n))
    (tau/2 Delta_h of Section 7.2 acting on the mode is -lam), the weights
    (b0, b1 = 1 - b0) of Eq. (FullyDiscreteDK) give (1 - b1 lam) / (1 + b0 lam):
    the symbol of A_h in Appendix C (Lemma Discrete_Energy_Est)."""
    lam = 2.0 * mu * (math.sin(math.pi * k[0] / n) ** 2 + math.sin(math.pi * k[1] / n) ** 2)
    return (1.0 - (1.0 - b0) * lam) / (1.0 + b0 * lam)


def closed_form_EP_cos1(length: float, n: int, tau: float, M: int, mass: float = 1.0, b0: float = 0.0) -> float:
    """E[P] for phi = cos(2 pi x1 / L) while rho stays positive, when the mean
    field minus its average is orthogonal to sin^2(2 pi x1 / L) at every step
    (e.g. rho0 = mass/L^2 (1 + a sin sin)).

    Lemma lem_Discrete_Martingale gives (rho^m, phi^m)_h as a martingale with
    phi^m = A_h^{M-m} I_h phi; the increment's conditional variance is
    N^-1 tau ([rho^m]^+, |nabla^c_h phi^{m+1}|^2)_h.  For this phi,
    |nabla^c_h phi^{m+1}|^2 = g^{2(M-m-1)} sin^2(2 pi x1/L) (sin(2 pi h/L)/h)^2,
    so E[P] = mass (tau/2)(sin(2 pi h/L)/h)^2 (1 - g^{2M}) / (1 - g^2) with
    g = 1 - 2 (tau/h^2) sin^2(pi/n).

    With b0 > 0 the noise of a step reaches rho through
    H = (I - b0 tau/2 Delta_h)^{-1}, so the increment pairs it with
    H phi^{m+1} = w phi^{m+1}, w = 1 / (1 + b0 lam), lam = 2 (tau/h^2) sin^2(pi/n),
    and g is the symbol (1 - b1 lam) / (1 + b0 lam): E[P] gains the factor w^2."""
    h = length / n
    mu = tau / (h * h)
    g = heat_symbol((1, 0), n, mu, b0)
    w = 1.0 / (1.0 + b0 * 2.0 * mu * math.sin(math.pi / n) ** 2)
    s = math.sin(2.0 * math.pi * h / length) / h
    return mass * 0.5 * tau * s * s * w * w * (1.0 - g ** (2 * M)) / (1.0 - g * g)
