"""ctypes binding of ``libmlmc_dk.so`` (C-ABI in include/mlmc_dk.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  There is no fallback: if the library is missing or no GPU is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmlmc_dk.so")

MAX_LEVELS = 16
MAX_OBS = 4
MAX_QUANT = 10
NSUM = 12

OK, NOT_CONVERGED = 0, 1
ERR_INVALID, ERR_CUDA, ERR_RANGE, ERR_UNSUPPORTED, ERR_STATE, ERR_TIMEOUT = -1, -2, -3, -4, -5, -6

_dp = ctypes.POINTER(ctypes.c_double)


class Config(ctypes.Structure):
    _fields_ = [
        ("length", ctypes.c_double),
        ("n0", ctypes.c_int32),
        ("L_max", ctypes.c_int32),
        ("T", ctypes.c_double),
        ("cfl_mu", ctypes.c_double),
        ("M0", ctypes.c_int32),
        ("N", ctypes.c_double),
        ("rho0", ctypes.POINTER(_dp)),
        ("n_obs", ctypes.c_int32),
        ("phi", ctypes.POINTER(_dp)),
        ("products", ctypes.c_int32),
        ("pilot", ctypes.c_int32),
        ("L_start", ctypes.c_int32),
        ("cuda_stream", ctypes.c_void_p),
        ("stream_from_n", ctypes.c_int32),
        ("theta_b0", ctypes.c_double),
        ("theta_kernel", ctypes.c_int32),
        ("coupling", ctypes.c_int32),
        ("state_repr", ctypes.c_int32),
    ]


class LevelDesc(ctypes.Structure):
    _fields_ = [
        ("level", ctypes.c_int32), ("n", ctypes.c_int32), ("M", ctypes.c_int32),
        ("h", ctypes.c_double), ("tau", ctypes.c_double),
        ("ybar_f", ctypes.c_double * MAX_OBS), ("ybar_c", ctypes.c_double * MAX_OBS),
        ("cost", ctypes.c_double), ("cost_mc", ctypes.c_double),
        ("next_sample", ctypes.c_int64), ("h2d_bytes", ctypes.c_int64), ("frac_bits", ctypes.c_int32),
        ("n_variants", ctypes.c_int32), ("variant_single", ctypes.c_int32), ("variant_coupled", ctypes.c_int32),
        ("lane_cols", ctypes.c_int32), ("lane_rows", ctypes.c_int32), ("cluster", ctypes.c_int32),
        ("streamed", ctypes.c_int32), ("in_flight", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
        ("split_capable", ctypes.c_int32), ("split_fraction", ctypes.c_double), ("batch_streamed", ctypes.c_int64),
        ("theta", ctypes.c_int32), ("theta_b0", ctypes.c_double), ("cheb_steps", ctypes.c_int32),
        ("coupling", ctypes.c_int32), ("fluct", ctypes.c_int32), ("band", ctypes.c_int32),
        ("bands", ctypes.c_int32), ("persistent", ctypes.c_int32), ("pdl", ctypes.c_int32),
    ]


class LevelSums(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [(k, ctypes.c_double) for k in (
        "dp1", "dp2", "dp3", "dp4", "pf1", "pf2", "pc1", "pc2", "yf1", "yf2", "yc1", "yc2",
        "max_mass_err", "cost", "wall_s", "kernel_s")] + [("launches", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Result(ctypes.Structure):
    _fields_ = [
        ("estimate", ctypes.c_double), ("variance", ctypes.c_double), ("eps_abs", ctypes.c_double),
        ("L", ctypes.c_int32), ("converged", ctypes.c_int32),
        ("M", ctypes.c_int64 * MAX_LEVELS),
        ("V", ctypes.c_double * MAX_LEVELS), ("E", ctypes.c_double * MAX_LEVELS),
        ("C", ctypes.c_double * MAX_LEVELS),
        ("estimates", ctypes.c_double * MAX_QUANT),
        ("sample_steps", ctypes.c_double), ("cell_steps", ctypes.c_double), ("wall_s", ctypes.c_double),
        ("kernel_s", ctypes.c_double * MAX_LEVELS), ("var_pf", ctypes.c_double * MAX_LEVELS),
        ("launches", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64),
    ]


# callbacks of mlmc_dk_algorithm1
ROUND_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double))
REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                             ctypes.c_int64)

_LIB = None


def lib() -> ctypes.CDLL:
    """Load the library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2311_08872_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.mlmc_dk_init.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
        L.mlmc_dk_free.argtypes = [vp]
        L.mlmc_dk_free.restype = None
        L.mlmc_dk_last_error.argtypes = [vp]
        L.mlmc_dk_last_error.restype = ctypes.c_char_p
        L.mlmc_dk_level_info.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(LevelDesc)]
        L.mlmc_dk_run_level.argtypes = [vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.POINTER(LevelSums)]
        L.mlmc_dk_run_mc.argtypes = [vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.POINTER(LevelSums)]
        L.mlmc_dk_run_level_dev.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_uint64, vp, vp, vp]
        L.mlmc_dk_estimate.argtypes = [vp, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(Result)]
        L.mlmc_dk_plan.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), _dp, _dp, _dp, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]
        L.mlmc_dk_mean_field_host.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                              _dp, _dp]
        L.mlmc_dk_mean_field_theta_host.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                                    ctypes.c_int64, ctypes.c_double, _dp, _dp]
        L.mlmc_dk_plan_ratio.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), _dp, _dp, _dp, ctypes.c_double,
                                         ctypes.c_double, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]
        _fp = ctypes.POINTER(ctypes.c_float)
        L.mlmc_dk_chebyshev_schedule_host.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_int32), _fp, _fp]
        L.mlmc_dk_fourier_restriction_host.argtypes = [ctypes.c_int32, _fp]
        L.mlmc_dk_save_state.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
        L.mlmc_dk_load_state.argtypes = [vp, vp, ctypes.c_size_t]
        L.mlmc_dk_num_quantities.argtypes = [vp]
        L.mlmc_dk_num_quantities.restype = ctypes.c_int32
        L.mlmc_dk_version.restype = ctypes.c_char_p
        L.mlmc_dk_run_level_static.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                               ctypes.c_int64, ctypes.c_uint64, vp, vp, vp, vp]
        L.mlmc_dk_algorithm1.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _dp,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ROUND_FN, REDUCE_FN, vp, ctypes.POINTER(Result)]
        L.mlmc_dk_band_wait_test.argtypes = [vp, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int32]
        L.mlmc_dk_stream_wait_test.argtypes = [vp, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int32]
        L.mlmc_dk_run_batch_dev.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, ctypes.c_uint64,
                                            vp, vp]
        L.mlmc_dk_run_batch.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.c_uint64, ctypes.POINTER(LevelSums)]
        L.mlmc_dk_batch_level_ms.argtypes = [vp, _dp]
        fp = ctypes.POINTER(ctypes.c_float)
        L.mlmc_dk_surrogate_init.argtypes = [vp, ctypes.c_uint64]
        L.mlmc_dk_surrogate_params.argtypes = [vp, fp, fp]
        L.mlmc_dk_surrogate_features.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                                 ctypes.c_uint64, fp]
        L.mlmc_dk_surrogate_forward.argtypes = [vp, fp, ctypes.c_int64, fp]
        L.mlmc_dk_surrogate_loss_grad.argtypes = [vp, fp, fp, ctypes.c_int32, _dp, fp]
        L.mlmc_dk_surrogate_train.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                              ctypes.c_uint64, _dp, _dp, _dp]
        L.mlmc_dk_run_surrogate.argtypes = [vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                            ctypes.POINTER(LevelSums)]
        L.mlmc_dk_estimate_surrogate.argtypes = [vp, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64,
                                                 ctypes.POINTER(Result), ctypes.POINTER(LevelSums)]
        L.mlmc_dk_set_variant.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.mlmc_dk_tune.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
        L.mlmc_dk_noise_dev.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                        ctypes.c_int32, ctypes.c_int32, vp, vp, vp]
        _LIB = L
    return _LIB


class MLMCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mlmc_dk error {code}: {msg}")
        self.code = code


def _check(rc: int, ctx=None, allow=(OK,)) -> int:
    if rc not in allow:
        msg = lib().mlmc_dk_last_error(ctx)
        raise MLMCError(rc, msg.decode() if msg else "")
    return rc


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------ host helpers
def mean_field_host(n: int, h: float, tau: float, M: int, rho0: np.ndarray, b0: float = 0.0) -> np.ndarray:
    r = _f64(rho0).reshape(-1)
    out = np.empty_like(r)
    if b0 == 0.0:
        _check(lib().mlmc_dk_mean_field_host(n, h, tau, M, r.ctypes.data_as(_dp), out.ctypes.data_as(_dp)))
    else:
        _check(lib().mlmc_dk_mean_field_theta_host(n, h, tau, M, b0, r.ctypes.data_as(_dp), out.ctypes.data_as(_dp)))
    return out.reshape(n, n)


def chebyshev_schedule(alpha: float):
    """(K, c1[:K], c2[:K]) of the theta-scheme's implicit solve (host logic)."""
    K = ctypes.c_int32(0)
    c1 = (ctypes.c_float * 64)()
    c2 = (ctypes.c_float * 64)()
    _check(lib().mlmc_dk_chebyshev_schedule_host(alpha, ctypes.byref(K), c1, c2))
    return K.value, np.array(c1[:K.value], dtype=np.float32), np.array(c2[:K.value], dtype=np.float32)


def fourier_restriction(n: int) -> np.ndarray:
    """The Fourier coupling's restriction matrix P1 [n/3][n] (host logic)."""
    P1 = np.zeros((n // 3, n), dtype=np.float32)
    _check(lib().mlmc_dk_fourier_restriction_host(n, P1.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return P1


def noise_dev(seed: int, level: int, stream_tag: int, sample: int, m: int, n: int,
              z_ptr: int = 0, raw_ptr: int = 0, stream: int = 0):
    """Normals / raw Philox words of one fine step into device memory."""
    _check(lib().mlmc_dk_noise_dev(seed, level, stream_tag, sample, m, n, ctypes.c_void_p(z_ptr or None),
                                   ctypes.c_void_p(raw_ptr or None), ctypes.c_void_p(stream or None)))


def algorithm1(run_round, reduce, L_max: int, n_quant: int, cost: Sequence[float], eps: float, *,
               ratio: float = 2.0, relative: bool = True, pilot: int = 256, L_start: int = 2, rank: int = 0,
               world: int = 1) -> Result:
    """mlmc_dk_algorithm1: Algorithm 1 (Section 7.1) in the library with this
    process's share of every round run by run_round(L, first, count) -> numpy
    sums [(L_max + 1), 2 + 12 n_quant] and the round's sums combined over the
    processes by reduce(sums) -> sums (used when world > 1)."""
    stride = 2 + NSUM * n_quant
    nl = L_max + 1
    errors = []

    def _round(_user, L, first, count, sums):
        try:
            f = [first[l] for l in range(nl)]
            c = [count[l] for l in range(nl)]
            out = np.asarray(run_round(int(L), f, c), dtype=np.float64).reshape(nl, stride)
            ctypes.memmove(sums, out.ctypes.data, out.nbytes)
            return 0
        except Exception as e:           # reported after the call
            errors.append(e)
            return 1

    def _reduce(_user, sums, n_levels, width):
        try:
            arr = np.ctypeslib.as_array(sums, shape=(int(n_levels) * int(width),)).copy()
            red = np.asarray(reduce(arr.reshape(int(n_levels), int(width))), dtype=np.float64)
            ctypes.memmove(sums, red.ctypes.data, red.nbytes)
            return 0
        except Exception as e:
            errors.append(e)
            return 1

    rf, df = ROUND_FN(_round), REDUCE_FN(_reduce)
    c = (ctypes.c_double * nl)(*[float(x) for x in cost])
    r = Result()
    rc = lib().mlmc_dk_algorithm1(L_max, L_start, pilot, n_quant, c, ratio, eps, int(relative), rank, world, rf, df,
                                  None, ctypes.byref(r))
    if errors:
        raise errors[0]
    _check(rc, None, allow=(OK, NOT_CONVERGED))
    return r


def plan(n: Sequence[int], s1: Sequence[float], s2: Sequence[float], cost: Sequence[float], eps: float,
         ratio: float = 2.0):
    """Algorithm 1's host step: targets by Eq. (opt_M_ell), stopping test of
    Eq. (convergence_criterion) for levels refining by `ratio`."""
    L = len(n) - 1
    n_ = (ctypes.c_int64 * (L + 1))(*n)
    a = (ctypes.c_double * (L + 1))(*s1)
    b = (ctypes.c_double * (L + 1))(*s2)
    c = (ctypes.c_double * (L + 1))(*cost)
    t = (ctypes.c_int64 * (L + 1))()
    conv = ctypes.c_int32(0)
    if ratio == 2.0:
        _check(lib().mlmc_dk_plan(L, n_, a, b, c, eps, t, ctypes.byref(conv)))
    else:
        _check(lib().mlmc_dk_plan_ratio(L, n_, a, b, c, eps, ratio, t, ctypes.byref(conv)))
    return list(t), bool(conv.value)


# ------------------------------------------------------------------ context
class Context:
    """An initialised MLMC context (levels, tables and buffers on the GPU)."""

    def __init__(self, length: float, n0: int, L_max: int, T: float, mu: float, N: float,
                 rho0: List[np.ndarray], phi: List[List[np.ndarray]], products: bool = False,
                 M0: int = 0, pilot: int = 0, L_start: int = 0, stream: Optional[int] = None,
                 stream_from_n: int = 0, theta_b0: float = 0.0, theta_kernel: bool = False, coupling: int = 0,
                 state_repr: int = 0):
        self._ctx = None
        self._rho0 = [_f64(r).reshape(-1) for r in rho0]
        self.n_obs = len(phi[0])
        self._phi = [_f64(p).reshape(-1) for lvl in phi for p in lvl]
        rho_ptrs = (_dp * len(self._rho0))(*[r.ctypes.data_as(_dp) for r in self._rho0])
        phi_ptrs = (_dp * len(self._phi))(*[p.ctypes.data_as(_dp) for p in self._phi])
        self.cfg = Config(length, n0, L_max, T, mu, M0, N, rho_ptrs, self.n_obs, phi_ptrs,
                          int(products), pilot, L_start, stream, stream_from_n, float(theta_b0),
                          int(theta_kernel), int(coupling), int(state_repr))
        h = ctypes.c_void_p()
        _check(lib().mlmc_dk_init(ctypes.byref(self.cfg), ctypes.byref(h)))
        self._ctx = h
        self.L_max = L_max
        self.n_quant = lib().mlmc_dk_num_quantities(self._ctx)

    @classmethod
    def from_workload(cls, wl, **kw) -> "Context":
        kw.setdefault("theta_b0", getattr(wl, "b0", 0.0))
        kw.setdefault("coupling", getattr(wl, "coupling", 0))
        return cls(wl.length, wl.n0, wl.L_max, wl.T, wl.mu, wl.N, wl.rho0_all(), wl.phi_all(),
                   products=wl.products, M0=wl.M0, **kw)

    def close(self):
        if self._ctx is not None:
            lib().mlmc_dk_free(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._ctx

    def level_info(self, level: int) -> LevelDesc:
        d = LevelDesc()
        _check(lib().mlmc_dk_level_info(self._ctx, level, ctypes.byref(d)), self._ctx)
        return d

    def run_level(self, level: int, n_samples: int, seed: int, sums=None, mc: bool = False):
        if sums is None:
            sums = (LevelSums * self.n_quant)()
        fn = lib().mlmc_dk_run_mc if mc else lib().mlmc_dk_run_level
        _check(fn(self._ctx, level, n_samples, seed, sums), self._ctx)
        return sums

    def run_level_dev(self, level: int, stream_tag: int, first: int, n_samples: int, seed: int,
                      sums_ptr: int, samples_ptr: int = 0, stream: int = 0):
        """Device-resident batch; pointers are device addresses (e.g. tensor.data_ptr())."""
        _check(lib().mlmc_dk_run_level_dev(self._ctx, level, stream_tag, first, n_samples, seed,
                                           ctypes.c_void_p(sums_ptr), ctypes.c_void_p(samples_ptr or None),
                                           ctypes.c_void_p(stream or None)), self._ctx)

    def run_level_static(self, level: int, stream_tag: int, first: int, n_samples: int, seed: int,
                         sums_ptr: int, samples_ptr: int = 0, err_ptr: int = 0, stream: int = 0):
        """As run_level_dev, with the scratch in the library's static device array
        (no allocation; calls must not overlap on the GPU)."""
        _check(lib().mlmc_dk_run_level_static(self._ctx, level, stream_tag, first, n_samples, seed,
                                              ctypes.c_void_p(sums_ptr), ctypes.c_void_p(samples_ptr or None),
                                              ctypes.c_void_p(err_ptr or None), ctypes.c_void_p(stream or None)),
               self._ctx)

    def band_wait_test(self, level: int, polls: int, stall_band: int) -> int:
        """Failure-detection test of the band kernel's bounded waits; returns the status code."""
        return lib().mlmc_dk_band_wait_test(self._ctx, level, polls, stall_band)

    def stream_wait_test(self, level: int, polls: int, stall_tile: int) -> int:
        """Failure-detection test of the persistent streamed kernel's bounded waits; returns the status code."""
        return lib().mlmc_dk_stream_wait_test(self._ctx, level, polls, stall_tile)

    def run_batch_dev(self, counts, first: int, seed: int, sums_ptr: int, stream: int = 0):
        """All levels concurrently (CUDA graph); sums_ptr: device double[L_max+1][sums_len]."""
        c = (ctypes.c_int64 * (self.L_max + 1))(*[int(x) for x in counts])
        _check(lib().mlmc_dk_run_batch_dev(self._ctx, c, first, seed, ctypes.c_void_p(sums_ptr),
                                           ctypes.c_void_p(stream or None)), self._ctx)

    def batch_level_ms(self):
        ms = (ctypes.c_double * (self.L_max + 1))()
        _check(lib().mlmc_dk_batch_level_ms(self._ctx, ms), self._ctx)
        return list(ms)

    def set_batch_split(self, level: int, fraction: float):
        """Share of `level`'s batch samples run on the streamed kernels beside the graph."""
        _check(lib().mlmc_dk_set_batch_split(self._ctx, level, ctypes.c_double(fraction)), self._ctx)

    def tune_batch(self, counts, repeats: int = 1):
        """Time the batch `counts` for a few split fractions and keep the fastest;
        returns (fraction, seconds spent)."""
        c = (ctypes.c_int64 * (self.L_max + 1))(*[int(x) for x in counts])
        f, t = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(lib().mlmc_dk_tune_batch(self._ctx, c, repeats, ctypes.byref(f), ctypes.byref(t)), self._ctx)
        return f.value, t.value

    def run_batch(self, counts, seed: int):
        """Host form: returns sums[level][quantity]."""
        c = (ctypes.c_int64 * (self.L_max + 1))(*[int(x) for x in counts])
        sums = (LevelSums * ((self.L_max + 1) * self.n_quant))()
        _check(lib().mlmc_dk_run_batch(self._ctx, c, seed, sums), self._ctx)
        return [[sums[l * self.n_quant + q] for q in range(self.n_quant)] for l in range(self.L_max + 1)]

    # ---- learned level below level 0
    N_PARAMS = 148481            # parameters of the one-output network (148224 + 257 K in general)

    def surrogate_init(self, seed: int = 0):
        _check(lib().mlmc_dk_surrogate_init(self._ctx, seed), self._ctx)

    def surrogate_info(self):
        """(parameters, outputs) of the initialised network."""
        p, k = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(lib().mlmc_dk_surrogate_info(self._ctx, ctypes.byref(p), ctypes.byref(k)), self._ctx)
        return p.value, k.value

    def surrogate_params(self, theta=None) -> np.ndarray:
        fp = ctypes.POINTER(ctypes.c_float)
        out = np.empty(self.surrogate_info()[0], dtype=np.float32)
        tin = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib().mlmc_dk_surrogate_params(self._ctx, out.ctypes.data_as(fp),
                                              None if tin is None else tin.ctypes.data_as(fp)), self._ctx)
        return out

    def surrogate_features(self, first: int, n: int, seed: int, stream_tag: int = 0, direct: bool = False):
        fp = ctypes.POINTER(ctypes.c_float)
        X = np.empty((n, 64), dtype=np.float32)
        _check(lib().mlmc_dk_surrogate_features(self._ctx, int(direct), stream_tag, first, n, seed,
                                                X.ctypes.data_as(fp)), self._ctx)
        return X

    def surrogate_forward(self, X) -> np.ndarray:
        fp = ctypes.POINTER(ctypes.c_float)
        X = np.ascontiguousarray(X, dtype=np.float32)
        K = self.surrogate_info()[1]
        y = np.empty((X.shape[0], K), dtype=np.float32)
        _check(lib().mlmc_dk_surrogate_forward(self._ctx, X.ctypes.data_as(fp), X.shape[0], y.ctypes.data_as(fp)),
               self._ctx)
        return y[:, 0] if K == 1 else y

    def surrogate_loss_grad(self, X, T):
        fp = ctypes.POINTER(ctypes.c_float)
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        P, K = self.surrogate_info()
        if T.size != X.shape[0] * K:
            raise ValueError(f"targets must have {K} value(s) per row")
        g = np.empty(P, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        _check(lib().mlmc_dk_surrogate_loss_grad(self._ctx, X.ctypes.data_as(fp), T.ctypes.data_as(fp), X.shape[0],
                                                 ctypes.byref(loss), g.ctypes.data_as(fp)), self._ctx)
        return loss.value, g

    def surrogate_train(self, n_pairs: int, epochs: int, batch: int, lr: float, seed: int):
        a, b, c = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(lib().mlmc_dk_surrogate_train(self._ctx, n_pairs, epochs, batch, lr, seed, ctypes.byref(a),
                                             ctypes.byref(b), ctypes.byref(c)), self._ctx)
        return {"train_mse": a.value, "val_mse": b.value, "seconds": c.value}

    def run_surrogate(self, part: int, n: int, seed: int, sums=None):
        """Sums of n samples of the level below 0 (part -1) or of the correction
        level (part 0), one LevelSums per quantity."""
        if sums is None:
            sums = (LevelSums * self.n_quant)()
        _check(lib().mlmc_dk_run_surrogate(self._ctx, part, n, seed, sums), self._ctx)
        return sums

    def estimate_surrogate(self, eps: float, relative: bool, seed: int):
        r, s = Result(), LevelSums()
        _check(lib().mlmc_dk_estimate_surrogate(self._ctx, eps, int(relative), seed, ctypes.byref(r), ctypes.byref(s)),
               self._ctx, allow=(OK, NOT_CONVERGED))
        return r, s

    def set_variant(self, level: int, coupled: bool, variant: int):
        _check(lib().mlmc_dk_set_variant(self._ctx, level, int(coupled), variant), self._ctx)

    def tune(self, repeats: int = 1) -> float:
        """Time every kernel variant per level and keep the fastest; returns seconds spent."""
        t = ctypes.c_double(0.0)
        _check(lib().mlmc_dk_tune(self._ctx, repeats, ctypes.byref(t)), self._ctx)
        return t.value

    def variants(self):
        """[(variant_single, variant_coupled)] per level."""
        return [(d.variant_single, d.variant_coupled) for d in (self.level_info(l) for l in range(self.L_max + 1))]

    def estimate(self, eps: float, relative: bool, seed: int) -> Result:
        r = Result()
        _check(lib().mlmc_dk_estimate(self._ctx, eps, int(relative), seed, ctypes.byref(r)), self._ctx,
               allow=(OK, NOT_CONVERGED))
        return r

    def save_state(self) -> bytes:
        n = ctypes.c_size_t(0)
        _check(lib().mlmc_dk_save_state(self._ctx, None, ctypes.byref(n)), self._ctx)
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().mlmc_dk_save_state(self._ctx, buf, ctypes.byref(n)), self._ctx)
        return buf.raw[: n.value]

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().mlmc_dk_load_state(self._ctx, buf, len(blob)), self._ctx)


def sample_stride(n_obs: int) -> int:
    """Doubles per sample in run_level_dev's per-sample output."""
    return 2 * n_obs + 2


def sums_len(n_quant: int) -> int:
    return 2 + NSUM * n_quant
