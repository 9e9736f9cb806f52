"""GB300-native shifted-Laplace-preconditioned FGMRES for the heterogeneous
Helmholtz equation (Kazemi, arXiv 1712.08740).

The solver is the CUDA library ``lib/libhelm.so`` behind ``include/helm.h``;
``helm`` is its ctypes binding. Importing ``helm`` fails if the library has
not been built (``build.build()``): there is no CPU fallback.
"""
__all__ = ["build", "helm"]
