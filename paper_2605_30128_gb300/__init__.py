"""GB300 (sm_103a) R-ChFSI filter for the noncollinear / spin-orbit finite-element
Kohn-Sham eigenproblem H X = M X Lambda (arXiv 2605.30128).

The computation lives in librchfsi.so (CUDA, C ABI in include/rchfsi.h);
``rchfsi`` is its ctypes binding with the same names, ``problem`` sets up a
synthetic workload through it, ``autograd`` wraps the filter adjoint.
"""
from .build import build, LIB
from . import rchfsi

__all__ = ["build", "LIB", "rchfsi"]
