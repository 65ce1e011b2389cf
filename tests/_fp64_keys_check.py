"""Run as a module in its own process: a build of the library whose FP32
key-error bound is so large that every rule-based column of the mixed form
takes the in-kernel FP64-key path (warp kernels and the large-tile CTA
kernel), compared with the oracle like the mixed parity tests.  Exit status 0
when every case is at parity."""
import sys

import numpy as np
import torch

import oracle as O
from paper_1208_3573_gb300 import build, diaf
from tests._parity import assert_parity, compare, host_factors
from tests._problems import random_sparse
from workloads import make_workload, pattern_of, upper_budget


def run(A, PW, vrule, budget, alg, tie_tol=O.TIE_TOL):
    dA = diaf.DeviceCSC.from_host(A)
    dP = diaf.DeviceCSC.from_host(PW)
    dB = None if budget is None else torch.from_numpy(np.ascontiguousarray(budget, np.int32)).cuda()
    F = diaf.factor(dA, dP, vrule, dB, None, alg=alg, prec="mixed32", tie_tol=tie_tol)
    torch.cuda.synchronize()
    return F


def main() -> int:
    diaf.LIB_PATH = build.build(variant="fp64keys", extra=["-DDIAF_MIXED_DELTA_SCALE=1e9"])
    cases = []
    for name in ("helmholtz40", "lognormal16", "powerlaw6k"):
        w = make_workload(name)
        cases += [(name, w.A, w.PW, w.vrule, w.budget, w.tie_tol)]
    for cplx in (False, True):
        A = random_sparse(300, 0.015, 17, cplx)
        cases += [(f"random{'C' if cplx else 'R'}", A, pattern_of(A), O.RULE_UPPER, upper_budget(A), O.TIE_TOL)]
    failed = 0
    for name, A, PW, vrule, budget, tie_tol in cases:
        for alg in "SQ":
            g = host_factors(run(A, PW, vrule, budget, alg, tie_tol))
            o = O.factor(A, PW, vrule, budget, alg=alg, tie_tol=tie_tol)
            rep = compare(g, o, A, PW, alg, rtol_res=1e-4, vec_tol=1e-6, mixed=True, floor_rel=1e-10)
            try:
                assert_parity(rep)
                print(name, alg, "ok")
            except AssertionError as e:
                failed += 1
                print(name, alg, "FAIL", str(e)[:600])
    return 1 if failed else 0


if __name__ == "__main__":
    sys.exit(main())
