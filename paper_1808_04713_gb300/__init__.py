"""GB300-native dual-primal domain-decomposition spectral-element Helmholtz solver.

The solver lives in the native library ``libddh.so`` (C ABI declared in ``include/ddh.h``):
host C++ setup and factorisation plus hand-written sm_103a CUDA kernels.  ``ddh`` is a thin
ctypes binding with the same names; PyTorch only provides device memory and streams.
"""
from .ddh import DDH, DDHError, Options, load_library  # noqa: F401
