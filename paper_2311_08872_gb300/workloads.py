"""Seeded synthetic workloads for the 2-D Dean--Kawasaki MLMC hot path.

This module only describes inputs: torus size, level-0 grid, final time, CFL
ratio, particle number, the initial mean-field profile rho0 sampled at grid
points (the pointwise interpolation I_h of Section 2), the test functions phi
sampled at grid points, and seeds.  It holds none of the scheme's arithmetic
(no stepping, no noise, no observables, no level coupling), so that the CUDA
path and the FP64 oracle can both be fed from it without sharing method code.

Grid convention: point (i1, i2) of an n x n grid sits at ((i1+o)*h, (i2+o)*h)
with h = L/n and the workload's offset o; arrays are row-major with flat index
i1*n + i2.  With o = 0 the coarse point I of a level pair is the fine point 2I
and its coupled noise block {2I, 2I+1}^2 lies to its right (the Right-Most
coupling of Section 3.2; the paper's grid {-pi, ..., pi-h}^2 is this point set
when n is even).  With o = 1/2 (cell-centred points, the shifted grid of
Remark avoid_right_bias) the coarse point (I+1/2)*2h is the centre of the same
block: the symmetric variant of the coupling, with no change to the kernels.

Workloads:
  * ``mc32``         -- plain MC on 32^2, unit torus, T=0.01, N=1e4.
  * ``mlmc16_256``   -- coupled MLMC, levels 16^2..256^2, T=0.02, N=1e5.
  * ``mlmc16_256_sym`` -- the same on cell-centred grids (symmetric coupling).
  * ``lowdens32_512``-- low-density periodised Gaussian, levels 32^2..512^2.
  * ``large32_1024`` -- levels 32^2..1024^2, T=0.05, N=1e6, four cosine modes
                        plus all pairwise products.
  * ``paper_reg`` / ``paper_irreg`` -- the paper's Section 7 setting on
                        (0, 2pi)^2 with levels 4^2..128^2 (h_l = 2pi 2^-(2+l),
                        tau_l = 1e-3 4^(5-l), T = 1.024, phi = sin x + sin y).
  * ``theta16_64``   -- Crank--Nicolson weights b0 = b1 = 1/2 of Eq.
                        (FullyDiscreteDK) at tau/h^2 = 1 (twice the explicit
                        limit), levels 16^2..64^2, T=0.02, N=1e5.
  * ``theta16_128``  -- the same weights and step ratio on levels 16^2..128^2.
  * ``implicit16_64``-- implicit Euler weights b0 = 1, b1 = 0 at tau/h^2 = 2,
                        same grids.
  * ``fourier6_54``  -- Fourier coupling (Section 3.1), levels 6^2, 18^2, 54^2
                        (h ratio 3, tau ratio 9), T=0.02, N=1e5.
  * ``fourier6_162`` -- the same with a fourth level, 162^2 (a 6-CTA cluster
                        per sample).
  * ``paper_reg_fourier`` -- the paper's regular setting (Section 7.2) with the
                        Fourier coupling on 6^2, 18^2, 54^2 (same tau/h^2 as the
                        paper's levels).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

TWO_PI = 2.0 * math.pi


def grid_coords(n: int, length: float, offset: float = 0.0) -> Tuple[np.ndarray, np.ndarray]:
    """(x1, x2) coordinate arrays of shape (n, n) for the n x n torus grid,
    points at (i + offset) h."""
    h = length / n
    i = (np.arange(n, dtype=np.float64) + offset) * h
    return np.meshgrid(i, i, indexing="ij")


# ---------------------------------------------------------------- rho0 kinds
def rho0_sinsin(x1, x2, length, amp=0.5):
    w = TWO_PI / length
    return 1.0 + amp * np.sin(w * x1) * np.sin(w * x2)


def rho0_sinsin_cos(x1, x2, length):
    w = TWO_PI / length
    return 1.0 + 0.5 * np.sin(w * x1) * np.sin(w * x2) + 0.3 * np.cos(2.0 * w * x2)


def rho0_gauss(x1, x2, length, base=0.02, peak=0.98, width=0.02, centre=(0.5, 0.5)):
    """base + peak * exp(-|x - centre|^2 / width), periodised over image shifts."""
    out = np.full_like(x1, base)
    for s1 in (-1, 0, 1):
        for s2 in (-1, 0, 1):
            d1 = x1 - centre[0] * length + s1 * length
            d2 = x2 - centre[1] * length + s2 * length
            out += peak * np.exp(-(d1 * d1 + d2 * d2) / width)
    return out


def _paper_profile(x1, x2, reg: bool):
    s = np.sin(x1 - math.pi / 2) ** 2 + np.sin(x2 - 3 * math.pi / 2) ** 2
    if reg:
        return 1.0 + np.exp(-s / 2.0) / math.sqrt(TWO_PI)
    return np.exp(-s / (2.0 * 0.1))


_PAPER_Z: Dict[bool, float] = {}


def paper_normaliser(reg: bool, quad_n: int = 512) -> float:
    """Z such that the paper's profile / Z has unit mass on (0, 2pi)^2.

    The profile is smooth and periodic, so the periodic trapezoid rule on a
    512^2 grid is exact to rounding.
    """
    if reg not in _PAPER_Z:
        x1, x2 = grid_coords(quad_n, TWO_PI)
        h = TWO_PI / quad_n
        _PAPER_Z[reg] = float(np.sum(_paper_profile(x1, x2, reg)) * h * h)
    return _PAPER_Z[reg]


def rho0_paper(x1, x2, length, reg=True):
    return _paper_profile(x1, x2, reg) / paper_normaliser(reg)


RHO0_KINDS: Dict[str, Callable] = {
    "sinsin": rho0_sinsin,
    "sinsin_cos": rho0_sinsin_cos,
    "gauss": rho0_gauss,
    "paper_reg": lambda x1, x2, L: rho0_paper(x1, x2, L, reg=True),
    "paper_irreg": lambda x1, x2, L: rho0_paper(x1, x2, L, reg=False),
}


# ----------------------------------------------------------------- phi kinds
def phi_cos(x1, x2, length, k=(1, 0)):
    w = TWO_PI / length
    return np.cos(w * (k[0] * x1 + k[1] * x2))


def phi_sin_plus_sin(x1, x2, length):
    w = TWO_PI / length
    return np.sin(w * x1) + np.sin(w * x2)


@dataclass(frozen=True)
class Observable:
    kind: str                    # "cos" or "sin+sin"
    k: Tuple[int, int] = (1, 0)  # wave vector for "cos"

    def grid(self, n: int, length: float, offset: float = 0.0) -> np.ndarray:
        x1, x2 = grid_coords(n, length, offset)
        if self.kind == "cos":
            return phi_cos(x1, x2, length, self.k)
        if self.kind == "sin+sin":
            return phi_sin_plus_sin(x1, x2, length)
        raise ValueError(self.kind)


@dataclass
class Workload:
    name: str
    length: float
    n0: int
    L_max: int
    T: float
    mu: float                      # nominal CFL ratio tau/h^2
    N: float                       # particle number
    rho0_kind: str
    observables: List[Observable]
    products: bool = False
    seed: int = 0
    eps_rel: Optional[float] = None
    samples: Optional[int] = None   # fixed sample count (plain MC workload)
    M0: int = 0                     # >0 overrides M_0 = ceil(T / (mu h0^2))
    alloc: Optional[Tuple[int, ...]] = None   # fixed per-level sample counts of one benchmark step
    alloc_scale: int = 1            # the eps-optimal allocation is about alloc * alloc_scale
    alloc_learned: Optional[Tuple[int, int]] = None  # with the learned level: (level below 0, correction level)
                                    # counts of one step, in place of alloc[0]
    offset: float = 0.0             # grid points at (i + offset) h: 0 right-most, 1/2 symmetric coupling
    b0: float = 0.0                 # implicit weight of the time step (b1 = 1 - b0); 0 explicit Euler--Maruyama
    coupling: int = 0               # 0 Right-Most NN (h ratio 2), 1 Fourier (h ratio 3)
    note: str = ""

    @property
    def ratio(self) -> int:
        return 3 if self.coupling == 1 else 2

    def n(self, level: int) -> int:
        return self.n0 * self.ratio ** level

    def rho0(self, level: int) -> np.ndarray:
        n = self.n(level)
        x1, x2 = grid_coords(n, self.length, self.offset)
        return np.ascontiguousarray(RHO0_KINDS[self.rho0_kind](x1, x2, self.length), dtype=np.float64)

    def phi(self, level: int) -> List[np.ndarray]:
        n = self.n(level)
        return [np.ascontiguousarray(o.grid(n, self.length, self.offset), dtype=np.float64)
                for o in self.observables]

    def rho0_all(self) -> List[np.ndarray]:
        return [self.rho0(l) for l in range(self.L_max + 1)]

    def phi_all(self) -> List[List[np.ndarray]]:
        return [self.phi(l) for l in range(self.L_max + 1)]

    def with_(self, **kw) -> "Workload":
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)


COS1 = Observable("cos", (1, 0))

WORKLOADS: Dict[str, Workload] = {
    "mc32": Workload("mc32", 1.0, 32, 0, 0.01, 0.1, 1e4, "sinsin", [COS1],
                     seed=0, samples=1000,
                     note="plain single-level MC, 32^2, 1000 samples"),
    "mlmc16_256": Workload("mlmc16_256", 1.0, 16, 4, 0.02, 0.1, 1e5, "sinsin", [COS1],
                           seed=1, eps_rel=1e-3, alloc=(578250, 28946, 4617, 1570, 955), alloc_scale=1024,
                           note="coupled MLMC, levels 16^2..256^2"),
    "mlmc16_256_sym": Workload("mlmc16_256_sym", 1.0, 16, 4, 0.02, 0.1, 1e5, "sinsin", [COS1],
                               seed=1, eps_rel=1e-3, alloc=(578250, 28946, 4617, 1570, 955), alloc_scale=1024,
                               offset=0.5,
                               note="mlmc16_256 on cell-centred grids: symmetric NN coupling"),
    "lowdens32_512": Workload("lowdens32_512", 1.0, 32, 4, 0.02, 0.1, 1e5, "gauss", [COS1],
                              seed=2, eps_rel=2e-3,
                              note="low-density periodised Gaussian, levels 32^2..512^2"),
    # alloc: the eps-optimal allocation for eps = 5e-4 relative (max over the 10
    # quantities of Eq. opt_M_ell, from pilot variances and device times per
    # sample on a GB300), divided by 2^20; alloc_learned: the same with the
    # learned level below 0 for levels {below 0, correction}
    "large32_1024": Workload("large32_1024", 1.0, 32, 5, 0.05, 0.1, 1e6, "sinsin_cos",
                             [Observable("cos", (1, 0)), Observable("cos", (0, 1)),
                              Observable("cos", (1, 1)), Observable("cos", (2, 0))],
                             products=True, seed=4, eps_rel=5e-4,
                             alloc=(12372, 566, 73, 17, 8, 5), alloc_scale=1 << 20, alloc_learned=(132504, 506),
                             note="levels 32^2..1024^2, four modes plus products"),
    "paper_reg": Workload("paper_reg", TWO_PI, 4, 5, 1.024, 1.024 / (TWO_PI / 4) ** 2, 2e9,
                          "paper_reg", [Observable("sin+sin")], seed=5, M0=1,
                          note="Section 7 setting, regular initial datum"),
    "paper_irreg": Workload("paper_irreg", TWO_PI, 4, 5, 1.024, 1.024 / (TWO_PI / 4) ** 2, 2e9,
                            "paper_irreg", [Observable("sin+sin")], seed=6, M0=1,
                            note="Section 7 setting, irregular initial datum"),
    "theta16_64": Workload("theta16_64", 1.0, 16, 2, 0.02, 1.0, 1e5, "sinsin", [COS1],
                           seed=7, eps_rel=1e-2, b0=0.5,
                           note="Crank-Nicolson weights at tau/h^2 = 1, levels 16^2..64^2"),
    "theta16_128": Workload("theta16_128", 1.0, 16, 3, 0.02, 1.0, 1e5, "sinsin", [COS1],
                            seed=7, eps_rel=1e-2, b0=0.5,
                            note="Crank-Nicolson weights at tau/h^2 = 1, levels 16^2..128^2 (128^2 on 4-CTA clusters)"),
    "implicit16_64": Workload("implicit16_64", 1.0, 16, 2, 0.02, 2.0, 1e5, "sinsin", [COS1],
                              seed=8, eps_rel=1e-2, b0=1.0,
                              note="implicit Euler weights at tau/h^2 = 2, levels 16^2..64^2"),
    "fourier6_54": Workload("fourier6_54", 1.0, 6, 2, 0.02, 0.1, 1e5, "sinsin", [COS1],
                            seed=9, eps_rel=1e-2, coupling=1,
                            note="Fourier coupling, levels 6^2, 18^2, 54^2"),
    "fourier6_162": Workload("fourier6_162", 1.0, 6, 3, 0.02, 0.1, 1e5, "sinsin", [COS1],
                             seed=9, eps_rel=1e-2, coupling=1,
                             note="Fourier coupling, levels 6^2, 18^2, 54^2, 162^2 (162^2 on 6-CTA clusters)"),
    "paper_reg_fourier": Workload("paper_reg_fourier", TWO_PI, 6, 2, 1.024, 1.024 / (TWO_PI / 4) ** 2, 2e9,
                                  "paper_reg", [Observable("sin+sin")], seed=10, coupling=1,
                                  note="Section 7 setting, regular datum, Fourier coupling on 6^2, 18^2, 54^2"),
}


def get(name: str) -> Workload:
    return WORKLOADS[name]
