"""Seeded synthetic inputs for the columnwise DIAF setup.

This package holds only input generation: the test operators, their sparsity
patterns (the standard matrix subspaces of Byckling & Huhtanen, Sec. 2) and
the named workload configurations.  It contains none of the method's
arithmetic, so both the CPU oracle and the CUDA path may import it.
"""
from .csc import CSC, Pattern
from .operators import convdiff2d, helmholtz2d, powerlaw_random, lognormal3d
from .patterns import pattern_of, pattern_power, upper_budget, lower_budget, diagonal_pattern
from .configs import Workload, make_workload, WORKLOADS

__all__ = [
    "CSC", "Pattern", "convdiff2d", "helmholtz2d", "powerlaw_random", "lognormal3d",
    "pattern_of", "pattern_power", "upper_budget", "lower_budget", "diagonal_pattern",
    "Workload", "make_workload", "WORKLOADS",
]
