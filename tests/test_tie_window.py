"""The tie window of the V rule on the symmetric Helmholtz stencil.

Sec. 3.1 picks the admissible rows of largest leverage.  On the compact
9-point stencil mirrored rows have equal leverage, which the computed keys
reproduce only to rounding, so the rule needs a tie window; the workload uses
tau = 1e-3 (wide enough for FP32 keys to resolve the exact ties).  This test
pins that the wide window selects the same I_j as a window at the rounding
level (1e-12) on every column of the full-size 512 x 512 operator: the
selection cut never falls between keys closer than 1e-3, so the window only
orders exact ties, as the paper's largest-norm rule intends.  (Measured on
the operator: mirrored keys agree to 5e-16, the smallest distinct gap is
7e-4 but never at the cut, where distinct keys are at least 0.7 apart.)"""
import numpy as np

import oracle as O
from workloads import make_workload


def test_helmholtz_tie_window_changes_no_selection():
    w = make_workload("helmholtz512")
    assert w.tie_tol == 1e-3
    wide = O.factor(w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=w.tie_tol)
    for tau in (1e-12, 1e-9):
        tight = O.factor(w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=tau)
        assert np.array_equal(wide.voff, tight.voff)
        assert np.array_equal(wide.Vrowidx, tight.Vrowidx)
