"""Python binding of libdiaf.so (include/diaf.h): argument marshalling only.

Every computation runs in the CUDA library.  PyTorch provides device memory
and streams; outputs owned by the library are exposed to PyTorch as
zero-copy views (through __cuda_array_interface__) that keep their factor
handle alive.  There is no CPU path: a missing library or GPU raises.

Typical use (A in CSC, int32 indices, float64 or complex128 values)::

    from paper_1208_3573_gb300 import diaf
    A  = diaf.DeviceCSC.from_host(A_host)                 # or DeviceCSC(n, colptr, rowidx, vals)
    PW = diaf.DeviceCSC.from_host(W_pattern_host)         # the W pattern, e.g. pattern(A^2)
    l  = torch.full((n,), 3, dtype=torch.int32, device="cuda")   # entries per column of V
    F  = diaf.factor(A, PW, diaf.RULE_UPPER, l, alg="S", prec="mixed32")
    F.W, F.V, F.res, F.flags                              # CSC factors, per-column residuals, flags
    y  = F.apply(x)                                       # y = W V^-1 x
    S  = diaf.Solver(A)
    x, info = S.bicgstab(b, F, tol=1e-8)                  # or S.gmres(b, F, tol=1e-6, restart=50)

Variants: alg "Q" (unit v_j) or "S" (unit w_j); prec "fp64" or "mixed32";
V by rule (RULE_UPPER / LOWER / ALL, or RULE_BLOCK with `blocks`) or a fixed
pattern (RULE_FIXED, Vfixed=...); stab_tol for the stabilised DIAF-Q;
Plan(...) for numeric refactorisation on new values of A by CUDA-graph
replay; autotune(...) for the launch tuning; sparsified_powers(...) for the
Neumann-series W pattern; propose_features / mlp_* / propose_select (and
learned.Proposer) for the learned W pattern.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdiaf.so")

DIAF_OK, DIAF_EINVAL, DIAF_ENOMEM, DIAF_ECUDA, DIAF_ENUMERIC, DIAF_ETIMEOUT, DIAF_EUNSUPPORTED = range(7)
DIAF_F64, DIAF_C128 = 0, 1
ALG = {"Q": 1, "S": 2}
PREC = {"fp64": 0, "mixed32": 1}
RULE_FIXED, RULE_UPPER, RULE_LOWER, RULE_ALL, RULE_BLOCK = 0, 1, 2, 3, 4
FLAG_RANK_DEFICIENT, FLAG_DEGENERATE, FLAG_VJJ_ZERO, FLAG_JACOBI_NOCONV = 1, 2, 4, 8
FLAG_NONFINITE, FLAG_EMPTY, FLAG_FP64_FALLBACK, FLAG_STABILISED = 16, 32, 64, 128


class DiafError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"diaf status {status}: {detail}")
        self.status = status


class CSC_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("colptr", ctypes.c_void_p),
                ("rowidx", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("dtype", ctypes.c_int32)]


class Pattern_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("colptr", ctypes.c_void_p),
                ("rowidx", ctypes.c_void_p)]


class VSpec_t(ctypes.Structure):
    _fields_ = [("rule", ctypes.c_int32), ("fixed", ctypes.POINTER(Pattern_t)), ("budget", ctypes.c_void_p),
                ("tie_tol", ctypes.c_double), ("stab_tol", ctypes.c_double), ("stab_r", ctypes.c_double),
                ("blocks", ctypes.c_void_p)]


class Tuning_t(ctypes.Structure):
    _fields_ = [("m_edge0", ctypes.c_int32), ("m_edge1", ctypes.c_int32), ("warps_per_block", ctypes.c_int32 * 2),
                ("small_tiles", ctypes.c_int32), ("large_tiles", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"m_edge0": self.m_edge0, "m_edge1": self.m_edge1, "warps_per_block": list(self.warps_per_block),
                "small_tiles": self.small_tiles, "large_tiles": self.large_tiles}

    @staticmethod
    def from_dict(d: dict | None) -> "Tuning_t | None":
        if d is None:
            return None
        w = d.get("warps_per_block", [0, 0])
        return Tuning_t(d.get("m_edge0", 0), d.get("m_edge1", 0), (ctypes.c_int32 * 2)(*w), d.get("small_tiles", 0),
                        d.get("large_tiles", 0))


class Info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("dtype", ctypes.c_int32), ("alg", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("nnz_w", ctypes.c_int64), ("nnz_v", ctypes.c_int64), ("max_k", ctypes.c_int32),
                ("max_m", ctypes.c_int32), ("max_l", ctypes.c_int32), ("n_buckets", ctypes.c_int32),
                ("bucket_cols", ctypes.c_int32 * 8)]


class SolveInfo_t(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32), ("breakdown", ctypes.c_int32),
                ("relres", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Loads libdiaf.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.diaf_factor.argtypes = [ctypes.POINTER(CSC_t), ctypes.POINTER(Pattern_t), ctypes.POINTER(VSpec_t),
                                  ctypes.c_int32, ctypes.c_int32, vp, ctypes.POINTER(vp)]
        L.diaf_factor_tuned.argtypes = [ctypes.POINTER(CSC_t), ctypes.POINTER(Pattern_t), ctypes.POINTER(VSpec_t),
                                        ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Tuning_t), vp,
                                        ctypes.POINTER(vp)]
        L.diaf_autotune.argtypes = [ctypes.POINTER(CSC_t), ctypes.POINTER(Pattern_t), ctypes.POINTER(VSpec_t),
                                    ctypes.c_int32, ctypes.c_int32, vp, ctypes.POINTER(Tuning_t),
                                    ctypes.POINTER(ctypes.c_float)]
        L.diaf_plan_create.argtypes = [ctypes.POINTER(CSC_t), ctypes.POINTER(Pattern_t), ctypes.POINTER(VSpec_t),
                                       ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Tuning_t), vp,
                                       ctypes.POINTER(vp)]
        L.diaf_plan_execute.argtypes = [vp, vp]
        L.diaf_plan_factors.argtypes = [vp]
        L.diaf_plan_factors.restype = vp
        L.diaf_plan_free.argtypes = [vp]
        L.diaf_plan_free.restype = None
        L.diaf_factor_info_get.argtypes = [vp, ctypes.POINTER(Info_t)]
        L.diaf_get_factors.argtypes = [vp, ctypes.POINTER(CSC_t), ctypes.POINTER(CSC_t),
                                       ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.diaf_apply.argtypes = [vp, vp, vp, vp]
        L.diaf_apply_static.argtypes = [vp, vp, vp, vp]
        L.diaf_sync.argtypes = [vp, vp]
        L.diaf_free.argtypes = [vp]
        L.diaf_free.restype = None
        L.diaf_solver_create.argtypes = [ctypes.POINTER(CSC_t), vp, ctypes.POINTER(vp)]
        L.diaf_solver_free.argtypes = [vp]
        L.diaf_solver_free.restype = None
        L.diaf_bicgstab.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_int32, vp, ctypes.POINTER(SolveInfo_t)]
        L.diaf_gmres.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, vp,
                                 ctypes.POINTER(SolveInfo_t)]
        L.diaf_factor_timings.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int32]
        L.diaf_launch_count.restype = ctypes.c_longlong
        L.diaf_apply_prep_counts.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.diaf_apply_prep_counts.restype = None
        L.diaf_set_device_memory_limit.argtypes = [ctypes.c_int64]
        L.diaf_device_memory_in_use.restype = ctypes.c_int64
        L.diaf_factor_fallbacks.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]
        L.diaf_propose_features.argtypes = [ctypes.POINTER(CSC_t), ctypes.POINTER(Pattern_t), vp, vp]
        L.diaf_mlp_forward.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
        L.diaf_mlp_grad.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp, vp]
        L.diaf_mlp_adam.argtypes = [vp, vp, vp, vp, ctypes.c_int32, ctypes.c_float, vp]
        L.diaf_propose_select.argtypes = [ctypes.POINTER(Pattern_t), vp, ctypes.c_int32, vp, vp, vp]
        L.diaf_scaled_residuals.argtypes = [vp, vp, vp]
        L.diaf_toggle_targets.argtypes = [ctypes.POINTER(Pattern_t), vp, vp, vp, ctypes.c_int32, ctypes.c_double,
                                          vp, vp]
        L.diaf_release_pool_memory.argtypes = []
        L.diaf_sparsified_count.argtypes = [ctypes.POINTER(CSC_t), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            vp, ctypes.POINTER(ctypes.c_int64), vp]
        L.diaf_sparsified_fill.argtypes = [ctypes.POINTER(CSC_t), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           vp, vp, vp]
        L.diaf_level_schedule.argtypes = [ctypes.c_int32, vp, vp, vp, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]
        L.diaf_status_string.argtypes = [ctypes.c_int]
        L.diaf_status_string.restype = ctypes.c_char_p
        L.diaf_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(st: int) -> None:
    if st != DIAF_OK:
        L = lib()
        raise DiafError(st, f"{L.diaf_status_string(st).decode()}: {L.diaf_last_error().decode()}")


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous()
    return t.data_ptr()


@dataclass
class DeviceCSC:
    """A matrix or pattern in CSC on the GPU (int32 indices; float64 or complex128 values)."""

    n: int
    colptr: torch.Tensor
    rowidx: torch.Tensor
    vals: torch.Tensor | None = None

    @property
    def nnz(self) -> int:
        return int(self.rowidx.numel())

    @property
    def dtype_code(self) -> int:
        return DIAF_C128 if (self.vals is not None and self.vals.is_complex()) else DIAF_F64

    def csc_t(self) -> CSC_t:
        return CSC_t(self.n, self.nnz, _ptr(self.colptr), _ptr(self.rowidx), _ptr(self.vals), self.dtype_code)

    def pattern_t(self) -> Pattern_t:
        return Pattern_t(self.n, self.nnz, _ptr(self.colptr), _ptr(self.rowidx))

    @staticmethod
    def from_host(M, device="cuda", pin=False) -> "DeviceCSC":
        """M: workloads.CSC or workloads.Pattern (numpy arrays)."""
        def to(a):
            t = torch.from_numpy(a)
            if pin:
                t = t.pin_memory()
            return t.to(device, non_blocking=pin)
        vals = getattr(M, "vals", None)
        return DeviceCSC(M.n, to(M.colptr), to(M.rowidx), None if vals is None else to(vals))


class _CAI:
    """__cuda_array_interface__ view of library-owned memory; holds `owner`."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}
        self._owner = owner


def _view(ptr, count, typestr, owner, torch_dtype):
    if count == 0 or not ptr:
        return torch.empty(0, dtype=torch_dtype, device="cuda")
    return torch.as_tensor(_CAI(ptr, (count,), typestr, owner), device="cuda")


class _Handle:
    """Owns one diaf_factors* (freed when the last view or Factors drops it),
    or borrows it from an owner kept alive here (a plan's factors)."""

    def __init__(self, ptr: int, owner=None):
        self.ptr = ctypes.c_void_p(ptr)
        self.owner = owner

    def free(self):
        if self.ptr.value and self.owner is None:
            lib().diaf_free(self.ptr)
        self.ptr = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Factors:
    """W, V (CSC, library-owned device memory), per-column residuals and flags.

    The tensors are zero-copy views of the library's buffers; they keep the
    handle alive.  close() frees the buffers at once (the views must not be
    used afterwards)."""

    def __init__(self, handle: int, stream: int, owner=None):
        self._own = _Handle(handle, owner)
        self._stream = stream
        L = lib()
        info = Info_t()
        _check(L.diaf_factor_info_get(self._own.ptr, ctypes.byref(info)))
        self.info = info
        W = CSC_t(); V = CSC_t(); res = ctypes.c_void_p(); fl = ctypes.c_void_p()
        _check(L.diaf_get_factors(self._own.ptr, ctypes.byref(W), ctypes.byref(V), ctypes.byref(res),
                                  ctypes.byref(fl)))
        n = info.n
        cplx = W.dtype == DIAF_C128
        vt, vtd = ("<c16", torch.complex128) if cplx else ("<f8", torch.float64)
        o = self._own
        self.n = n
        self.W = DeviceCSC(n, _view(W.colptr, n + 1, "<i4", o, torch.int32),
                           _view(W.rowidx, W.nnz, "<i4", o, torch.int32), _view(W.vals, W.nnz, vt, o, vtd))
        self.V = DeviceCSC(n, _view(V.colptr, n + 1, "<i4", o, torch.int32),
                           _view(V.rowidx, V.nnz, "<i4", o, torch.int32), _view(V.vals, V.nnz, vt, o, vtd))
        self.res = _view(res.value, n, "<f8", o, torch.float64)
        self.flags = _view(fl.value, n, "<u4", o, torch.uint32)

    @property
    def handle(self):
        return self._own.ptr

    def timings(self) -> dict:
        """CUDA-event timings of the factorisation (ms): total, numeric, per bucket kernel."""
        buf = (ctypes.c_float * 10)()
        _check(lib().diaf_factor_timings(self._own.ptr, buf, 10))
        nb = self.info.n_buckets
        return {"total_ms": buf[0], "numeric_ms": buf[1], "bucket_ms": [buf[2 + b] for b in range(nb)],
                "bucket_cols": [self.info.bucket_cols[b] for b in range(nb)]}

    def fallbacks(self) -> list:
        """Mixed precision: columns per bucket computed by the FP64 path."""
        buf = (ctypes.c_int32 * 8)()
        _check(lib().diaf_factor_fallbacks(self._own.ptr, buf, 8))
        return [buf[b] for b in range(self.info.n_buckets)]

    def apply(self, x: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """y = W V^-1 x."""
        if y is None:
            y = torch.empty_like(x)
        _check(lib().diaf_apply(self._own.ptr, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def apply_static(self, x: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
        """y = W V^-1 x through diaf_apply_static: allocates nothing (y must be
        given; apply() must have run once on these factors)."""
        _check(lib().diaf_apply_static(self._own.ptr, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def sync(self, stream=None) -> None:
        _check(lib().diaf_sync(self._own.ptr, _stream(stream)))

    def close(self):
        self._own.free()


def launch_count() -> int:
    """Kernels launched by libdiaf.so in this process so far."""
    return int(lib().diaf_launch_count())


def apply_prep_counts() -> tuple:
    """(streamed, copied): apply preparations that built V's level schedule
    from V's structure streamed to the host during the numeric pass, and
    those that copied it after the pass."""
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    lib().diaf_apply_prep_counts(ctypes.byref(a), ctypes.byref(b))
    return int(a.value), int(b.value)


def set_device_memory_limit(nbytes: int) -> None:
    """Caps the device bytes the setup and apply paths may hold at once
    (0: no cap); a call that would exceed it raises DiafError (DIAF_ENOMEM)."""
    _check(lib().diaf_set_device_memory_limit(int(nbytes)))


def device_memory_in_use() -> int:
    """Device bytes the setup and apply paths hold now."""
    return int(lib().diaf_device_memory_in_use())


def release_pool_memory() -> None:
    """Returns the unused memory of the library's pool on the current device."""
    _check(lib().diaf_release_pool_memory())


def _args(A, PW, vrule, budget, Vfixed, tie_tol, stab=(0.0, 2.0), blocks=None):
    a = A.csc_t()
    pw = PW.pattern_t()
    fixed = Vfixed.pattern_t() if Vfixed is not None else None
    vs = VSpec_t(vrule, ctypes.pointer(fixed) if fixed is not None else None, _ptr(budget), tie_tol,
                 float(stab[0]), float(stab[1]), _ptr(blocks))
    return a, pw, vs, fixed


def factor(A: DeviceCSC, PW: DeviceCSC, vrule: int = RULE_UPPER, budget: torch.Tensor | None = None,
           Vfixed: DeviceCSC | None = None, alg: str = "S", prec: str = "fp64", tie_tol: float = 1e-9,
           stream=None, tuning: dict | None = None, stab_tol: float = 0.0, stab_r: float = 2.0,
           blocks: torch.Tensor | None = None) -> Factors:
    """Columnwise W, V with A W ~ V (diaf_factor / diaf_factor_tuned); stab_tol > 0
    turns on the stabilised DIAF-Q; vrule RULE_BLOCK with `blocks` (int32 block
    of every row, non-decreasing) gives a block-diagonal V."""
    L = lib()
    a, pw, vs, _keep = _args(A, PW, vrule, budget, Vfixed, tie_tol, (stab_tol, stab_r), blocks)
    h = ctypes.c_void_p()
    s = _stream(stream)
    t = Tuning_t.from_dict(tuning)
    _check(L.diaf_factor_tuned(ctypes.byref(a), ctypes.byref(pw), ctypes.byref(vs), ALG[alg], PREC[prec],
                               ctypes.byref(t) if t is not None else None, s, ctypes.byref(h)))
    return Factors(h.value, s)


def autotune(A: DeviceCSC, PW: DeviceCSC, vrule: int = RULE_UPPER, budget: torch.Tensor | None = None,
             Vfixed: DeviceCSC | None = None, alg: str = "S", prec: str = "fp64", tie_tol: float = 1e-9,
             stream=None, stab_tol: float = 0.0, stab_r: float = 2.0) -> tuple[dict, float]:
    """Fastest launch tuning of the numeric pass (diaf_autotune) and its time in ms."""
    L = lib()
    a, pw, vs, _keep = _args(A, PW, vrule, budget, Vfixed, tie_tol, (stab_tol, stab_r))
    best = Tuning_t()
    ms = ctypes.c_float()
    _check(L.diaf_autotune(ctypes.byref(a), ctypes.byref(pw), ctypes.byref(vs), ALG[alg], PREC[prec],
                           _stream(stream), ctypes.byref(best), ctypes.byref(ms)))
    return best.as_dict(), float(ms.value)


class Plan:
    """Symbolic pass once, numeric pass captured in a CUDA graph
    (diaf_plan_create); execute() replays it on the current values of A."""

    def __init__(self, A: DeviceCSC, PW: DeviceCSC, vrule: int = RULE_UPPER, budget: torch.Tensor | None = None,
                 Vfixed: DeviceCSC | None = None, alg: str = "S", prec: str = "fp64", tie_tol: float = 1e-9,
                 stream=None, tuning: dict | None = None, stab_tol: float = 0.0, stab_r: float = 2.0):
        L = lib()
        self._inputs = (A, PW, budget, Vfixed)  # the plan reads these buffers by pointer
        a, pw, vs, _keep = _args(A, PW, vrule, budget, Vfixed, tie_tol, (stab_tol, stab_r))
        t = Tuning_t.from_dict(tuning)
        h = ctypes.c_void_p()
        s = _stream(stream)
        _check(L.diaf_plan_create(ctypes.byref(a), ctypes.byref(pw), ctypes.byref(vs), ALG[alg], PREC[prec],
                                  ctypes.byref(t) if t is not None else None, s, ctypes.byref(h)))
        self._h = h
        self.factors = Factors(L.diaf_plan_factors(h), s, owner=self)

    def execute(self, stream=None) -> Factors:
        _check(lib().diaf_plan_execute(self._h, _stream(stream)))
        return self.factors

    def __del__(self):
        try:
            if self._h.value:
                lib().diaf_plan_free(self._h)
        except Exception:
            pass


class Solver:
    """A prepared for the Krylov solvers (diaf_solver_create)."""

    def __init__(self, A: DeviceCSC, stream=None):
        self._A = A
        h = ctypes.c_void_p()
        _check(lib().diaf_solver_create(ctypes.byref(A.csc_t()), _stream(stream), ctypes.byref(h)))
        self._h = h

    def bicgstab(self, b: torch.Tensor, M: Factors | None = None, tol=1e-8, maxit=1000, x=None, stream=None):
        if x is None:
            x = torch.empty_like(b)
        info = SolveInfo_t()
        _check(lib().diaf_bicgstab(self._h, M.handle if M is not None else None, _ptr(b), _ptr(x), tol, maxit,
                                   _stream(stream), ctypes.byref(info)))
        return x, info

    def gmres(self, b: torch.Tensor, M: Factors | None = None, tol=1e-6, restart=50, maxit=2000, x=None,
              stream=None):
        if x is None:
            x = torch.empty_like(b)
        info = SolveInfo_t()
        _check(lib().diaf_gmres(self._h, M.handle if M is not None else None, _ptr(b), _ptr(x), tol, restart,
                                maxit, _stream(stream), ctypes.byref(info)))
        return x, info

    def __del__(self):
        try:
            if self._h.value:
                lib().diaf_solver_free(self._h)
        except Exception:
            pass


# ---------------------------------------------------------------- learned proposal of J_j
PROP_NFEAT, PROP_HIDDEN, PROP_NPARAM = 8, 32, 1377


def propose_features(A: DeviceCSC, CAND: DeviceCSC, stream=None) -> torch.Tensor:
    """[CAND.nnz, 8] float32 candidate features (diaf_propose_features)."""
    feat = torch.empty((CAND.nnz, PROP_NFEAT), dtype=torch.float32, device=A.colptr.device)
    a, c = A.csc_t(), CAND.pattern_t()
    _check(lib().diaf_propose_features(ctypes.byref(a), ctypes.byref(c), _ptr(feat), _stream(stream)))
    return feat


def mlp_forward(params: torch.Tensor, feat: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Scores of the network on every feature row (diaf_mlp_forward)."""
    assert params.dtype == torch.float32 and params.numel() == PROP_NPARAM and feat.dtype == torch.float32
    n = feat.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=feat.device)
    _check(lib().diaf_mlp_forward(_ptr(params), _ptr(feat), n, _ptr(out), _stream(stream)))
    return out


def mlp_grad(params: torch.Tensor, feat: torch.Tensor, target: torch.Tensor, grad: torch.Tensor | None = None,
             loss: torch.Tensor | None = None, stream=None):
    """(grad, loss) of the mean squared error (diaf_mlp_grad); loss stays on the device."""
    assert target.dtype == torch.float32 and target.numel() == feat.shape[0]
    if grad is None:
        grad = torch.empty(PROP_NPARAM, dtype=torch.float32, device=feat.device)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
    _check(lib().diaf_mlp_grad(_ptr(params), _ptr(feat), _ptr(target), feat.shape[0], _ptr(grad), _ptr(loss),
                               _stream(stream)))
    return grad, loss


def mlp_adam(params, grad, m, v, step: int, lr: float, stream=None) -> None:
    """One Adam step in place on params, m, v (diaf_mlp_adam)."""
    _check(lib().diaf_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), step, lr, _stream(stream)))


def propose_select(CAND: DeviceCSC, score: torch.Tensor, keep: int, stream=None) -> DeviceCSC:
    """Kept pattern (diagonal + best scores, at most `keep` per column) as a DeviceCSC pattern."""
    dev = CAND.colptr.device
    colptr = torch.empty(CAND.n + 1, dtype=torch.int32, device=dev)
    rowidx = torch.empty(max(1, min(CAND.nnz, CAND.n * keep)), dtype=torch.int32, device=dev)
    c = CAND.pattern_t()
    _check(lib().diaf_propose_select(ctypes.byref(c), _ptr(score), keep, _ptr(colptr), _ptr(rowidx),
                                     _stream(stream)))
    nnz = int(colptr[-1].item())
    return DeviceCSC(CAND.n, colptr, rowidx[:nnz].clone())


def scaled_residuals(F: "Factors", stream=None) -> torch.Tensor:
    """res_j / |V(j,j)| per column on the device (diaf_scaled_residuals)."""
    out = torch.empty(F.n, dtype=torch.float64, device=F.res.device)
    _check(lib().diaf_scaled_residuals(F._own.ptr, _ptr(out), _stream(stream)))
    return out


def toggle_targets(CAND: DeviceCSC, in_base: torch.Tensor, r0: torch.Tensor, rt: torch.Tensor, slot: int,
                   clip: float, value: torch.Tensor, stream=None) -> torch.Tensor:
    """Writes the toggle targets of candidate slot `slot` into value (diaf_toggle_targets)."""
    assert in_base.dtype == torch.uint8 and r0.dtype == rt.dtype == value.dtype == torch.float64
    c = CAND.pattern_t()
    _check(lib().diaf_toggle_targets(ctypes.byref(c), _ptr(in_base), _ptr(r0), _ptr(rt), int(slot), float(clip),
                                     _ptr(value), _stream(stream)))
    return value


def sparsified_powers(A: DeviceCSC, k: int = 2, p_l: int = 0, keep: int = 0, stream=None) -> DeviceCSC:
    """W pattern by sparsified powers (diaf_sparsified_count / _fill)."""
    L = lib()
    a = A.csc_t()
    s = _stream(stream)
    colptr = torch.empty(A.n + 1, dtype=torch.int32, device=A.colptr.device)
    nnz = ctypes.c_int64()
    _check(L.diaf_sparsified_count(ctypes.byref(a), k, p_l, keep, _ptr(colptr), ctypes.byref(nnz), s))
    rowidx = torch.empty(max(int(nnz.value), 1), dtype=torch.int32, device=A.colptr.device)
    _check(L.diaf_sparsified_fill(ctypes.byref(a), k, p_l, keep, _ptr(colptr), _ptr(rowidx), s))
    return DeviceCSC(A.n, colptr, rowidx[:int(nnz.value)])


def level_schedule(colptr, rowidx):
    """Host-side level schedule of a triangular V given by its columns (numpy
    int32 arrays): (level per row, number of levels, upper?).  No GPU call."""
    import numpy as np
    cp = np.ascontiguousarray(colptr, dtype=np.int32)
    ri = np.ascontiguousarray(rowidx, dtype=np.int32)
    n = cp.size - 1
    lev = np.zeros(max(n, 1), dtype=np.int32)
    nlev, up = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib().diaf_level_schedule(n, cp.ctypes.data, ri.ctypes.data if ri.size else None, lev.ctypes.data,
                                     ctypes.byref(nlev), ctypes.byref(up)))
    return lev[:n], int(nlev.value), bool(up.value)


def contiguous_blocks(n: int, size: int, device="cuda") -> torch.Tensor:
    """Block ids for DIAF_RULE_BLOCK: consecutive runs of `size` rows."""
    return (torch.arange(n, dtype=torch.int32, device=device) // size).contiguous()
