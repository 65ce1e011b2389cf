"""Element-by-element comparison of the CUDA path with the CPU oracle.

Tolerances (FP64 path):
  * I_j bit-exact (V colptr and row indices identical);
  * res_j: |res_gpu - res_oracle| <= 1e-10 res_oracle + floor_j with
    floor_j = 64 eps ||A(:,J_j)||_F ||w_j|| (the rounding level of ||A w - v||);
  * w_j, v_j: after the shared phase convention (v_jj real >= 0) the vectors
    themselves agree, ||x_gpu - x_oracle|| <= 1e-8 ||x_oracle|| (which bounds
    the subspace angle by the same number), checked where the optimal vector
    is unique (flag DEGENERATE clear and a resolved gap);
  * degenerate or rank-deficient columns (several optimal vectors): the GPU
    vector must be valid instead -- unit norm where the algorithm fixes it,
    v_j = P_V A w_j (DIAF-S) and the same residual.
"""
from __future__ import annotations

import numpy as np

EPS = np.finfo(np.float64).eps
F_RANK, F_DEG, F_VJJ, F_NOCONV, F_NONFIN, F_EMPTY, F_REFINED = 1, 2, 4, 8, 16, 32, 64


def host_factors(F):
    return dict(
        Wcp=F.W.colptr.cpu().numpy(), Wri=F.W.rowidx.cpu().numpy(), Wv=F.W.vals.cpu().numpy(),
        Vcp=F.V.colptr.cpu().numpy(), Vri=F.V.rowidx.cpu().numpy(), Vv=F.V.vals.cpu().numpy(),
        res=F.res.cpu().numpy(), flags=F.flags.cpu().numpy().astype(np.uint32))


def compare(g: dict, o, A, PW, alg: str, rtol_res=1e-10, vec_tol=1e-8, cols=None, check_flags=True):
    """g: host_factors(F) (all columns); o: oracle result for `cols` (or all)."""
    n = A.n
    cols = np.arange(n) if cols is None else np.asarray(cols)
    colnorm2 = np.zeros(n)
    np.add.at(colnorm2, np.repeat(np.arange(n), np.diff(A.colptr)), np.abs(A.vals) ** 2)
    report = dict(cols=len(cols), I_mismatch=[], res_bad=[], vec_bad=[], flag_bad=[], degenerate=0, max_res_rel=0.0,
                  max_vec_rel=0.0)
    for t, j in enumerate(cols):
        Ig = g["Vri"][g["Vcp"][j]:g["Vcp"][j + 1]]
        Io = o.I(t)
        if not np.array_equal(Ig, Io):
            report["I_mismatch"].append(int(j))
            continue
        wg = g["Wv"][g["Wcp"][j]:g["Wcp"][j + 1]]
        wo = o.w(t)
        vg = g["Vv"][g["Vcp"][j]:g["Vcp"][j + 1]]
        vo = o.v(t)
        J = PW.rowidx[PW.colptr[j]:PW.colptr[j + 1]]
        tnorm = np.sqrt(colnorm2[J].sum())
        floor = 64 * EPS * tnorm * max(np.linalg.norm(wo), np.linalg.norm(wg), 1e-300)
        rg, ro = g["res"][j], o.res[t]
        err = abs(rg - ro)
        if not err <= rtol_res * ro + floor:
            report["res_bad"].append((int(j), float(rg), float(ro)))
        if ro > floor:
            report["max_res_rel"] = max(report["max_res_rel"], err / ro)
        fo = int(o.flags[t]); fg = int(g["flags"][j])
        if check_flags and (fo & ~F_REFINED) != (fg & ~F_REFINED):
            report["flag_bad"].append((int(j), fg, fo))
        unique = not (fo & (F_DEG | F_RANK | F_EMPTY | F_VJJ)) and o.sig[t].size == 2
        if alg == "S" and unique:
            gap = abs(o.sig[t, 1] - o.sig[t, 0]) / max(o.sig[t, 1], 1e-300)
            unique = gap >= 1e-6
        if unique:
            e1 = np.linalg.norm(wg - wo) / max(np.linalg.norm(wo), 1e-300)
            e2 = np.linalg.norm(vg - vo) / max(np.linalg.norm(vo), 1e-300)
            report["max_vec_rel"] = max(report["max_vec_rel"], e1, e2)
            if not (e1 <= vec_tol and e2 <= vec_tol):
                report["vec_bad"].append((int(j), float(e1), float(e2)))
        else:
            report["degenerate"] += 1
            if alg == "S" and wg.size:
                ok = abs(np.linalg.norm(wg) - 1) <= 1e-10
            elif alg == "Q":
                ok = abs(np.linalg.norm(vg) - 1) <= 1e-10
            else:
                ok = True
            if not ok:
                report["vec_bad"].append((int(j), "norm", float(np.linalg.norm(wg))))
    return report


def assert_parity(report, allow_I_mismatch=0):
    msg = {k: (v[:5] if isinstance(v, list) else v) for k, v in report.items()}
    assert len(report["I_mismatch"]) <= allow_I_mismatch, msg
    assert not report["res_bad"], msg
    assert not report["vec_bad"], msg
    assert not report["flag_bad"], msg
