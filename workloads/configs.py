"""Named synthetic workloads for the columnwise setup.

Each workload fixes the operator A, the W pattern, the V specification
(a fixed pattern, or an admissibility rule plus a per-column budget l_j for
the optimal V-pattern rule of Sec. 3.1), the right-hand side b = A * ones
(the paper's choice of b, Sec. 5) and the default algorithm.

  convdiff2d   2D upwind convection-diffusion, W = pattern(A) or pattern(A^2)
  powerlaw     random power-law column degrees (uneven tile sizes)
  helmholtz2d  complex shifted 9-point Helmholtz
  lognormal3d  3D heterogeneous diffusion-convection (learned-proposal study)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .csc import CSC, Pattern
from . import operators as ops
from . import patterns as pats

RULE_UPPER, RULE_LOWER, RULE_ALL = 1, 2, 3


@dataclass
class Workload:
    name: str
    A: CSC
    PW: Pattern
    vrule: int = RULE_UPPER          # admissibility rule for the V pattern (0 = fixed)
    budget: np.ndarray | None = None  # l_j per column (diagonal included), None = all admissible
    Vfixed: Pattern | None = None
    alg: str = "S"                   # "S" (unit w_j, Sec. 2.2) or "Q" (unit v_j, Sec. 2.1)
    b: np.ndarray | None = None
    meta: dict = field(default_factory=dict)
    # leverage keys within tie_tol of the current largest count as tied in the
    # V rule (lower row wins); symmetric stencils have exact ties
    tie_tol: float = 1e-9

    @property
    def n(self) -> int:
        return self.A.n


def _finish(name, A, PW, alg, **meta) -> Workload:
    b = A.to_scipy() @ np.ones(A.n, dtype=A.vals.dtype)
    return Workload(name, A, PW, RULE_UPPER, pats.upper_budget(A), None, alg, b, meta)


def convdiff(N: int = 32, wpower: int = 1, alg: str = "S") -> Workload:
    A = ops.convdiff2d(N)
    PW = pats.pattern_of(A) if wpower == 1 else pats.pattern_power(A, wpower)
    return _finish(f"convdiff2d_{N}x{N}_Wp{wpower}", A, PW, alg, grid=N, wpower=wpower)


def powerlaw(n: int = 200_000, seed: int = 0, alg: str = "S") -> Workload:
    A = ops.powerlaw_random(n, seed)
    # the leverage rule can take every row of some W column into I_j, which
    # makes v_jj = 0 (V singular): this workload measures the setup only
    return _finish(f"powerlaw_n{n}_seed{seed}", A, pats.pattern_of(A), alg, seed=seed, apply=False)


def helmholtz(N: int = 512, alg: str = "S") -> Workload:
    k = ops.helmholtz_wavenumber(N)
    A = ops.helmholtz2d(N, k)
    w = _finish(f"helmholtz2d_{N}x{N}", A, pats.pattern_of(A), alg, grid=N, wavenumber=k)
    w.tie_tol = 1e-3  # the 9-point stencil is symmetric: mirrored rows tie exactly
    return w


def lognormal(N: int = 64, seed: int = 0, wpower: int = 2, alg: str = "S") -> Workload:
    A = ops.lognormal3d(N, seed=seed)
    PW = pats.pattern_power(A, wpower)
    return _finish(f"lognormal3d_{N}^3_seed{seed}_Wp{wpower}", A, PW, alg, grid=N, seed=seed, wpower=wpower)


# The five named configurations (full sizes) and small parity-size variants.
WORKLOADS = {
    "convdiff32": lambda **kw: convdiff(32, 1, **kw),            # n = 1,024,  W = pattern(A)
    "convdiff256_A2": lambda **kw: convdiff(256, 2, **kw),       # n = 65,536, W = pattern(A^2)
    "powerlaw200k": lambda **kw: powerlaw(200_000, 0, **kw),     # n = 200,000
    "helmholtz512": lambda **kw: helmholtz(512, **kw),           # n = 262,144, complex
    "lognormal64": lambda **kw: lognormal(64, 0, **kw),          # n = 262,144, candidates pattern(A^2)
    # parity-size variants (the oracle finishes these in seconds)
    "convdiff48_A2": lambda **kw: convdiff(48, 2, **kw),
    "powerlaw6k": lambda **kw: powerlaw(6_000, 0, **kw),
    "helmholtz40": lambda **kw: helmholtz(40, **kw),
    "lognormal16": lambda **kw: lognormal(16, 0, **kw),
}


def make_workload(name: str, **kw) -> Workload:
    return WORKLOADS[name](**kw)
