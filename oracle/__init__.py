"""CPU oracle for the columnwise DIAF setup -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check of __graft_entry__ and the CPU-baseline leg of
bench.py may import this package.  It shares no code with the CUDA library.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import factor, vcount, column, householder_qr, jacobi_svd, bicgstab, gmres, Preconditioner  # noqa: F401
