"""Exact solve u = H^-1 f by sparse LU (Eq. 4), complex128.

This is the paper's "LU factorization" arm (Example section, Fig. 3a and
Fig. 6a). SuperLU through scipy does the factorisation.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .operator import assemble_H, assemble_M

__all__ = ["lu_solve", "lu_factor_H", "lu_factor_M", "true_relative_residual"]


def lu_factor_H(n, h, m, omega, alpha):
    return spla.splu(assemble_H(n, h, m, omega, alpha).tocsc())


def lu_factor_M(n, h, m, omega, alpha, beta1, beta2):
    return spla.splu(assemble_M(n, h, m, omega, alpha, beta1, beta2).tocsc())


def lu_solve(n, h, m, omega, alpha, f) -> np.ndarray:
    """u = H^-1 f for one right-hand side (array shaped like ``f``)."""
    lu = lu_factor_H(n, h, m, omega, alpha)
    return lu.solve(np.asarray(f, dtype=np.complex128).ravel()).reshape(np.shape(f))


def true_relative_residual(H, f, u) -> float:
    """||f - H u||_2 / ||f||_2 in complex128."""
    f = np.asarray(f).ravel()
    r = f - H @ np.asarray(u).ravel()
    return float(np.linalg.norm(r) / np.linalg.norm(f))
