"""GB300 (sm_103a) library for the columnwise construction of W, V with
A W ~ V -- direct approximate factoring of the inverse (Byckling & Huhtanen)
-- and for applying A^-1 ~ W V^-1 as a right preconditioner.

The computation lives in libdiaf.so (CUDA, C ABI in include/diaf.h); this
package is its thin binding (`diaf`) and build script (`build`).
"""
from . import diaf  # noqa: F401
from .diaf import DeviceCSC, Factors, Solver, factor, DiafError  # noqa: F401
