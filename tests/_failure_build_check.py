"""Run as a module in its own process: a build of the library with the
Jacobi sweep limit at 1.  The setup still returns finite (w_j, v_j, res_j),
with JACOBI_NOCONV set on the columns whose Jacobi needed more than one
sweep.  Exit status 0 when every check holds."""
import sys

import numpy as np
import torch

from paper_1208_3573_gb300 import build, diaf
from tests._parity import F_NOCONV, F_NONFIN, host_factors
from workloads import make_workload


def run(w, alg, prec):
    F = diaf.factor(diaf.DeviceCSC.from_host(w.A), diaf.DeviceCSC.from_host(w.PW), w.vrule,
                    torch.from_numpy(w.budget).cuda(), alg=alg, prec=prec, tie_tol=w.tie_tol)
    F.sync()
    return F


def main() -> int:
    diaf.LIB_PATH = build.build(variant="failtest", extra=["-DDIAF_MAX_SWEEPS=1"])
    w = make_workload("lognormal16")
    for alg in ("S", "Q"):
        for prec in ("fp64", "mixed32"):
            g = host_factors(run(w, alg, prec))
            noconv = int(np.count_nonzero(g["flags"] & F_NOCONV))
            finite = all(np.isfinite(g[k]).all() for k in ("Wv", "Vv", "res"))
            print(alg, prec, "NOCONV columns", noconv, "finite", finite,
                  "NONFINITE", int(np.count_nonzero(g["flags"] & F_NONFIN)))
            if not finite or np.any(g["flags"] & F_NONFIN):
                return 1
            if prec == "fp64" and noconv == 0:
                return 2
    return 0


if __name__ == "__main__":
    sys.exit(main())
