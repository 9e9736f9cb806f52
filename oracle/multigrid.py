"""Geometric-multigrid V-cycle for the shifted Laplacian M (Eq. 6), plain numpy.

The paper applies P^-1 in Eq. 7 but does not say how. The GPU path applies it
with one V-cycle. This module writes that V-cycle out in its textbook steps,
so that each GPU kernel can be checked against it on its own:

* levels: node counts n_c = (n + 1) / 2 per axis while every axis is odd and
  at least 3 and the level has more than ``coarse_max`` nodes. Spacing
  doubles. The slowness is injected (coarse node = coincident fine node).
  Each level's M is rediscretised with the same boundary rows.
* smoother: damped Jacobi, u <- u + w D^-1 (b - M u), with D = diag(M).
* restriction: full weighting (tensor product of [1/4, 1/2, 1/4]). Fine
  nodes outside the grid are taken as mirror images of the nodes inside.
  This is the adjoint of interpolation in the inner product that halves
  each boundary row once per face, divided by 2^d.
* prolongation: multilinear interpolation (coarse nodes sit on even fine
  nodes).
* coarsest level: a dense direct solve.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .operator import assemble_M

__all__ = ["Level", "build_levels", "jacobi", "residual", "restrict", "prolong", "vcycle",
           "can_coarsen"]


@dataclass
class Level:
    n: tuple          # node counts, axis 0 fastest
    h: float
    m: np.ndarray     # slowness, shape n[::-1]
    M: object         # CSR matrix of the shifted Laplacian on this level

    @property
    def shape(self):
        return self.n[::-1]

    @property
    def diag(self):
        return self.M.diagonal()


def can_coarsen(n) -> bool:
    return all(k % 2 == 1 and k >= 3 for k in n)


def build_levels(n, h, m, omega, alpha, beta1, beta2, coarse_max=1500, max_levels=32):
    n = tuple(int(k) for k in n)
    m = np.asarray(m, dtype=np.float64).reshape(n[::-1])
    levels = []
    while True:
        levels.append(Level(n, h, m, assemble_M(n, h, m, omega, alpha, beta1, beta2)))
        if int(np.prod(n)) <= coarse_max or not can_coarsen(n) or len(levels) >= max_levels:
            break
        m = m[tuple(slice(None, None, 2) for _ in n)]
        n = tuple((k + 1) // 2 for k in n)
        h = 2.0 * h
    return levels


def residual(level: Level, u, b):
    """b - M u on one level (flat vectors)."""
    return b - level.M @ u


def jacobi(level: Level, u, b, w):
    """One damped-Jacobi sweep."""
    return u + w * (b - level.M @ u) / level.diag


def restrict(fine_n, r):
    """Full weighting with mirrored outside nodes; returns the coarse vector."""
    fine_n = tuple(int(k) for k in fine_n)
    a = np.asarray(r).reshape(fine_n[::-1])
    for ax in range(a.ndim):
        p = np.pad(a, [(1, 1) if k == ax else (0, 0) for k in range(a.ndim)], mode="reflect")
        sl = lambda s: tuple(s if k == ax else slice(None) for k in range(a.ndim))  # noqa: E731
        # coarse node i sits on fine node 2i (padded index 2i + 1)
        a = 0.25 * p[sl(slice(0, -2, 2))] + 0.5 * p[sl(slice(1, -1, 2))] + \
            0.25 * p[sl(slice(2, None, 2))]
    return a.ravel()


def prolong(coarse_n, e):
    """Multilinear interpolation from the coarse grid to the next finer one."""
    coarse_n = tuple(int(k) for k in coarse_n)
    a = np.asarray(e).reshape(coarse_n[::-1])
    for ax in range(a.ndim):
        nc = a.shape[ax]
        shp = list(a.shape)
        shp[ax] = 2 * nc - 1
        out = np.zeros(shp, dtype=a.dtype)
        sl = lambda s: tuple(s if k == ax else slice(None) for k in range(a.ndim))  # noqa: E731
        out[sl(slice(0, None, 2))] = a
        out[sl(slice(1, None, 2))] = 0.5 * (a[sl(slice(0, -1))] + a[sl(slice(1, None))])
        a = out
    return a.ravel()


def vcycle(levels, b, nu1=1, nu2=1, w=0.6, level=0):
    """One V(nu1, nu2) cycle from a zero initial guess: returns ~ M^-1 b."""
    L = levels[level]
    if level == len(levels) - 1:
        return np.linalg.solve(L.M.toarray(), b)
    u = np.zeros_like(b)
    for _ in range(nu1):
        u = jacobi(L, u, b, w)
    rc = restrict(L.n, residual(L, u, b))
    ec = vcycle(levels, rc, nu1, nu2, w, level + 1)
    u = u + prolong(levels[level + 1].n, ec)
    for _ in range(nu2):
        u = jacobi(L, u, b, w)
    return u
