"""CPU oracle for the columnwise DIAF setup (Python side).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline are the only users.  The per-column arithmetic lives in the plain-C
file diaf_oracle.c (Householder QR, leverage rule of Sec. 3.1, DIAF-S of
Sec. 2.2, DIAF-Q of Sec. 2.1, one-sided Jacobi SVD); this module only
marshals arrays through ctypes, and adds the solve-phase references
(W V^-1 x of eq. afac, BiCGSTAB and restarted GMRES) in plain numpy/scipy.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

RULE_FIXED, RULE_UPPER, RULE_LOWER, RULE_ALL, RULE_BLOCK = 0, 1, 2, 3, 4
ALG = {"Q": 1, "S": 2}
F_RANK_DEFICIENT, F_DEGENERATE, F_VJJ_ZERO, F_JACOBI_NOCONV, F_NONFINITE, F_EMPTY = 1, 2, 4, 8, 16, 32
F_STABILISED = 128
TIE_TOL = 1e-9  # leverage keys within this distance of the largest count as tied (lower row wins)

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_lib = None


def _load():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build())
        L.diaf_oracle_vcount.argtypes = [ctypes.c_int, _i32p, _i32p, _i32p, _i32p, ctypes.c_int, _i32p, _i32p,
                                         _i32p, _i32p, ctypes.c_int, _i32p, _i32p, ctypes.c_int]
        L.diaf_oracle_factor.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _i32p, _i32p, ctypes.c_int, _i32p,
                                         _i32p, _i32p, _i32p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, _i32p, _i64p,
                                         _f64p, _i32p, _f64p, _f64p, _u32p, _f64p, _f64p, ctypes.c_int]
        L.diaf_oracle_column.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _i32p, _i32p, ctypes.c_int, _i32p,
                                         _i32p, _i32p, _i32p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, _f64p, _i32p,
                                         _f64p, _f64p, _u32p, _f64p, _f64p, _i32p, _i32p, _f64p]
        L.diaf_oracle_qr.argtypes = [ctypes.c_int, ctypes.c_int, _f64p, _f64p, _f64p]
        L.diaf_oracle_jacobi_svd.argtypes = [ctypes.c_int, ctypes.c_int, _f64p, _f64p, _f64p]
        L.diaf_oracle_jacobi_svd.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _nthreads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


class _Inputs:
    """Keeps contiguous copies alive for the duration of a call."""

    def __init__(self, A, PW, vrule, budget, Vfixed, blocks=None):
        self.n = A.n
        self.Acp = np.ascontiguousarray(A.colptr, np.int32)
        self.Ari = np.ascontiguousarray(A.rowidx, np.int32)
        self.Av = np.ascontiguousarray(A.vals, np.complex128).view(np.float64)
        self.Wcp = np.ascontiguousarray(PW.colptr, np.int32)
        self.Wri = np.ascontiguousarray(PW.rowidx, np.int32)
        self.rule = int(vrule)
        if self.rule == RULE_FIXED:
            self.Vcp = np.ascontiguousarray(Vfixed.colptr, np.int32)
            self.Vri = np.ascontiguousarray(Vfixed.rowidx, np.int32)
        else:
            self.Vcp = self.Vri = None
        self.budget = None if budget is None else np.ascontiguousarray(budget, np.int32)
        if self.rule == RULE_BLOCK and blocks is None:
            raise ValueError("RULE_BLOCK needs the block of every row")
        self.blk = None if blocks is None else np.ascontiguousarray(blocks, np.int32)
        self.real = not np.iscomplexobj(A.vals)

    def head(self):
        return (self.n, _p(self.Acp, _i32p), _p(self.Ari, _i32p))

    def wv(self):
        return (_p(self.Wcp, _i32p), _p(self.Wri, _i32p), self.rule, _p(self.Vcp, _i32p), _p(self.Vri, _i32p),
                _p(self.budget, _i32p), _p(self.blk, _i32p))


@dataclass
class OracleResult:
    cols: np.ndarray          # listed columns
    Wcolptr: np.ndarray       # = PW colptr
    Wrowidx: np.ndarray
    Wvals: np.ndarray         # full length nnz(PW); only listed columns filled
    voff: np.ndarray          # int64 [ncols+1] offsets into Vrowidx/Vvals (list order)
    Vrowidx: np.ndarray
    Vvals: np.ndarray
    res: np.ndarray
    flags: np.ndarray
    margin: np.ndarray
    sig: np.ndarray           # [ncols, 2]: selected singular value and its neighbour
    n: int

    def w(self, t: int) -> np.ndarray:
        j = self.cols[t]
        return self.Wvals[self.Wcolptr[j]:self.Wcolptr[j + 1]]

    def I(self, t: int) -> np.ndarray:
        return self.Vrowidx[self.voff[t]:self.voff[t + 1]]

    def v(self, t: int) -> np.ndarray:
        return self.Vvals[self.voff[t]:self.voff[t + 1]]

    def W_csc(self):
        import scipy.sparse as sp
        return sp.csc_matrix((self.Wvals, self.Wrowidx, self.Wcolptr), shape=(self.n, self.n))

    def V_csc(self):
        """V as a scipy matrix (requires all columns, in order)."""
        import scipy.sparse as sp
        assert len(self.cols) == self.n and np.all(self.cols == np.arange(self.n))
        return sp.csc_matrix((self.Vvals, self.Vrowidx, self.voff), shape=(self.n, self.n))


def vcount(A, PW, vrule=RULE_UPPER, budget=None, Vfixed=None, cols=None, nthreads=None, blocks=None) -> np.ndarray:
    L = _load()
    x = _Inputs(A, PW, vrule, budget, Vfixed, blocks)
    cl = None if cols is None else np.ascontiguousarray(cols, np.int32)
    nc = A.n if cl is None else cl.size
    out = np.zeros(nc, np.int32)
    L.diaf_oracle_vcount(*x.head(), *x.wv(), nc, _p(cl, _i32p), _p(out, _i32p), _nthreads(nthreads))
    return out


def factor(A, PW, vrule=RULE_UPPER, budget=None, Vfixed=None, alg="S", tie_tol=TIE_TOL, cols=None,
           nthreads=None, stab_tol=0.0, stab_r=2.0, blocks=None) -> OracleResult:
    """Columnwise W, V (Sec. 2.1 / 2.2 with the V rule of Sec. 3.1) for the
    listed columns (all when cols is None).  stab_tol > 0 turns on the
    stabilised DIAF-Q of Sec. 3.2 (|v_jj| < stab_tol -> v_jj imposed as stab_r).
    vrule RULE_BLOCK: `blocks` gives the block of every row (block-diagonal V)."""
    L = _load()
    x = _Inputs(A, PW, vrule, budget, Vfixed, blocks)
    cl = np.arange(A.n, dtype=np.int32) if cols is None else np.ascontiguousarray(cols, np.int32)
    nc = cl.size
    lc = vcount(A, PW, vrule, budget, Vfixed, cl, nthreads, blocks)
    voff = np.zeros(nc + 1, np.int64)
    np.cumsum(lc, out=voff[1:])
    Wv = np.zeros(PW.nnz, np.complex128)
    Vri = np.zeros(int(voff[-1]), np.int32)
    Vv = np.zeros(int(voff[-1]), np.complex128)
    res = np.zeros(nc); flags = np.zeros(nc, np.uint32); margin = np.zeros(nc); sig = np.zeros((nc, 2))
    L.diaf_oracle_factor(*x.head(), _p(x.Av, _f64p), *x.wv(), ALG[alg], float(tie_tol), float(stab_tol),
                         float(stab_r), nc, _p(cl, _i32p),
                         _p(voff, _i64p), _p(Wv.view(np.float64), _f64p), _p(Vri, _i32p),
                         _p(Vv.view(np.float64), _f64p), _p(res, _f64p), _p(flags, _u32p), _p(margin, _f64p),
                         _p(sig, _f64p), _nthreads(nthreads))
    if x.real:
        assert not np.any(Wv.imag) and not np.any(Vv.imag)
        Wv = Wv.real.copy(); Vv = Vv.real.copy()
    return OracleResult(cl, x.Wcp, x.Wri, Wv, voff, Vri, Vv, res, flags, margin, sig, A.n)


@dataclass
class ColumnInfo:
    j: int
    rows: np.ndarray   # R_j
    h: np.ndarray      # leverage per row of R_j
    I: np.ndarray
    w: np.ndarray
    v: np.ndarray
    res: float
    flags: int
    margin: float
    sig: np.ndarray


def column(A, PW, j, vrule=RULE_UPPER, budget=None, Vfixed=None, alg="S", tie_tol=TIE_TOL, stab_tol=0.0,
           stab_r=2.0, blocks=None) -> ColumnInfo:
    L = _load()
    x = _Inputs(A, PW, vrule, budget, Vfixed, blocks)
    k = int(PW.colptr[j + 1] - PW.colptr[j])
    l = int(vcount(A, PW, vrule, budget, Vfixed, [j], blocks=blocks)[0])
    mcap = int(sum(A.colptr[c + 1] - A.colptr[c] for c in PW.rowidx[PW.colptr[j]:PW.colptr[j + 1]])) + 1
    w = np.zeros(max(k, 1), np.complex128); Ir = np.zeros(max(l, 1), np.int32); v = np.zeros(max(l, 1), np.complex128)
    res = ctypes.c_double(); fl = ctypes.c_uint32(); mg = ctypes.c_double(); sig = np.zeros(2)
    m = ctypes.c_int32(); rows = np.zeros(mcap, np.int32); h = np.zeros(mcap)
    L.diaf_oracle_column(*x.head(), _p(x.Av, _f64p), *x.wv(), ALG[alg], float(tie_tol), float(stab_tol),
                         float(stab_r), int(j),
                         _p(w.view(np.float64), _f64p), _p(Ir, _i32p), _p(v.view(np.float64), _f64p),
                         ctypes.byref(res), ctypes.byref(fl), ctypes.byref(mg), _p(sig, _f64p), ctypes.byref(m),
                         _p(rows, _i32p), _p(h, _f64p))
    mm = m.value
    return ColumnInfo(j, rows[:mm].copy(), h[:mm].copy(), Ir[:l].copy(), w[:k].copy(), v[:l].copy(), res.value,
                      fl.value, mg.value, sig)


def householder_qr(T: np.ndarray):
    """Thin Householder QR of the oracle (complex128). Returns (Q, R)."""
    L = _load()
    m, k = T.shape
    a = np.asfortranarray(T, np.complex128).copy(order="F")
    r = np.zeros((k, k), np.complex128, order="F")
    q = np.zeros((m, min(m, k)), np.complex128, order="F")
    L.diaf_oracle_qr(m, k, a.ctypes.data_as(_f64p), r.ctypes.data_as(_f64p), q.ctypes.data_as(_f64p))
    return q, r


def jacobi_svd(G: np.ndarray):
    """One-sided Jacobi of the oracle: returns (sigma, V, GV, sweeps)."""
    L = _load()
    p, q = G.shape
    g = np.asfortranarray(G, np.complex128).copy(order="F")
    v = np.zeros((q, q), np.complex128, order="F")
    s = np.zeros(q)
    sweeps = L.diaf_oracle_jacobi_svd(p, q, g.ctypes.data_as(_f64p), v.ctypes.data_as(_f64p), s.ctypes.data_as(_f64p))
    return s, v, g, sweeps


# ------------------------------------------------------------ solve phase
class Preconditioner:
    """x -> W V^-1 x (eq. afac), with V factored once by a sparse LU."""

    def __init__(self, W, V):
        import scipy.sparse as sp
        from scipy.sparse.linalg import splu
        self.W = sp.csr_matrix(W)
        self.lu = splu(sp.csc_matrix(V))

    def __call__(self, x):
        return self.W @ self.lu.solve(x)


def bicgstab(A, b, M=None, tol=1e-8, maxit=1000):
    """Right-preconditioned BiCGSTAB (van der Vorst), x0 = 0, stop when
    ||r|| <= tol ||r0||.  Returns (x, its, relres, status) with status
    'ok', 'maxit' (no convergence: dagger in the paper's tables) or
    'breakdown' (double dagger)."""
    M = M or (lambda x: x)
    x = np.zeros_like(b)
    r = b.copy()
    r0n = np.linalg.norm(r)
    if r0n == 0:
        return x, 0, 0.0, "ok"
    rh = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b); p = np.zeros_like(b)
    for it in range(1, maxit + 1):
        rho = np.vdot(rh, r)
        if rho == 0:
            return x, it, np.linalg.norm(r) / r0n, "breakdown"
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = M(p)
        v = A @ ph
        den = np.vdot(rh, v)
        if den == 0:
            return x, it, np.linalg.norm(r) / r0n, "breakdown"
        alpha = rho / den
        s = r - alpha * v
        if np.linalg.norm(s) <= tol * r0n:
            x = x + alpha * ph
            return x, it, np.linalg.norm(s) / r0n, "ok"
        sh = M(s)
        t = A @ sh
        tt = np.vdot(t, t)
        if tt == 0:
            return x, it, np.linalg.norm(s) / r0n, "breakdown"
        omega = np.vdot(t, s) / tt
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        if np.linalg.norm(r) <= tol * r0n:
            return x, it, np.linalg.norm(r) / r0n, "ok"
        if omega == 0:
            return x, it, np.linalg.norm(r) / r0n, "breakdown"
        rho_old = rho
    return x, maxit, np.linalg.norm(r) / r0n, "maxit"


def gmres(A, b, M=None, restart=50, tol=1e-6, maxit=2000):
    """Right-preconditioned restarted GMRES(restart), modified Gram-Schmidt,
    x0 = 0, stop when ||b - A x|| <= tol ||b||.  Returns (x, its, relres, status)."""
    M = M or (lambda x: x)
    n = b.size
    dt = np.result_type(b.dtype, np.complex128 if np.iscomplexobj(b) else np.float64)
    x = np.zeros(n, dt)
    bn = np.linalg.norm(b)
    if bn == 0:
        return x, 0, 0.0, "ok"
    its = 0
    r = b - A @ x
    while its < maxit:
        beta = np.linalg.norm(r)
        if beta <= tol * bn:
            return x, its, beta / bn, "ok"
        Vb = np.zeros((n, restart + 1), dt)
        H = np.zeros((restart + 1, restart), dt)
        Vb[:, 0] = r / beta
        g = np.zeros(restart + 1, dt); g[0] = beta
        cs = np.zeros(restart, dt); sn = np.zeros(restart, dt)
        Z = np.zeros((n, restart), dt)
        kk = 0
        for kk in range(restart):
            its += 1
            Z[:, kk] = M(Vb[:, kk])
            wv = A @ Z[:, kk]
            for i in range(kk + 1):
                H[i, kk] = np.vdot(Vb[:, i], wv)
                wv = wv - H[i, kk] * Vb[:, i]
            H[kk + 1, kk] = np.linalg.norm(wv)
            if H[kk + 1, kk] != 0:
                Vb[:, kk + 1] = wv / H[kk + 1, kk]
            for i in range(kk):
                tmp = np.conj(cs[i]) * H[i, kk] + np.conj(sn[i]) * H[i + 1, kk]
                H[i + 1, kk] = -sn[i] * H[i, kk] + cs[i] * H[i + 1, kk]
                H[i, kk] = tmp
            den = np.hypot(abs(H[kk, kk]), abs(H[kk + 1, kk]))
            cs[kk] = H[kk, kk] / den if den else 1.0
            sn[kk] = H[kk + 1, kk] / den if den else 0.0
            H[kk, kk] = np.conj(cs[kk]) * H[kk, kk] + np.conj(sn[kk]) * H[kk + 1, kk]
            H[kk + 1, kk] = 0
            g[kk + 1] = -sn[kk] * g[kk]
            g[kk] = np.conj(cs[kk]) * g[kk]
            if abs(g[kk + 1]) <= tol * bn or its >= maxit:
                break
        m = kk + 1
        y = np.linalg.solve(np.triu(H[:m, :m]), g[:m])
        x = x + Z[:, :m] @ y
        r = b - A @ x
    rn = np.linalg.norm(r)
    return x, its, rn / bn, "ok" if rn <= tol * bn else "maxit"
