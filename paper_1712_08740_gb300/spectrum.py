"""Spectra of the discrete Helmholtz operator H and of its shifted-Laplace
preconditioned form, for small models (the paper's Example section, Fig. 2;
Eq. 6 and Eq. 7).

The library applies the operators on the GPU: H (Eq. 3) and the
preconditioner the solver uses in place of M^-1 (Eq. 6) are applied to the N
unit vectors, one call each. The N columns come back to the host, where numpy
computes the eigenvalues of the dense N x N matrix, so N is limited to a few
thousand nodes.

With precond="exact" the preconditioner is the dense inverse of M. The
right-preconditioned operator H M^-1 of Eq. 7 is then similar to M^-1 H
(M^-1 (H M^-1) M = M^-1 H), so the two have the same eigenvalues. With
precond="mg" it is H B, where B is the V-cycle. That is the operator the
solver actually iterates with, which the paper does not show.

`shift_sweep` repeats this for a list of shifts (beta1, beta2) of
M = -Lap - (beta1 - j beta2) w^2 m^2. For each shift it reports where the
spectrum lies and how many FGMRES iterations the solve takes. This is the
comparison behind the paper's choice of shift: its literal beta = (1, 1) is
(beta1, beta2) = (-1, 1) in this convention.
"""
from __future__ import annotations

import numpy as np

from . import helm

__all__ = ["dense_operator", "eigenvalues", "summarize", "shift_sweep"]

MAX_NODES = 4096


def _columns(N, apply):
    """The N x N matrix whose column i is apply(e_i)."""
    A = np.empty((N, N), dtype=np.complex128)
    e = np.zeros(N, dtype=np.complex128)
    y = np.empty(N, dtype=np.complex128)
    for i in range(N):
        e[i] = 1.0
        apply(e, y)
        A[:, i] = y
        e[i] = 0.0
    return A


def dense_operator(grid, which="preconditioned"):
    """Dense matrix of an operator of `grid` (a helm.Grid with model and
    shift set), built from the library's GPU operators.

    which: "H" (Eq. 3), "M" (the shifted Laplacian on the fine level, Eq. 6) or
    "preconditioned" (H P, P the grid's preconditioner: M^-1 for
    precond="exact", one V-cycle for "mg", the identity for "none").
    """
    N = grid.N
    if N > MAX_NODES:
        raise ValueError(f"{N} nodes: dense spectra are for grids of at most {MAX_NODES} nodes")
    if which == "H":
        return _columns(N, grid.apply_H)
    if which == "M":
        return _columns(N, lambda x, y: grid.apply_M(0, x, y))
    if which == "preconditioned":
        z = np.empty(N, dtype=np.complex128)

        def hp(x, y):
            grid.apply_precond(x, z)
            grid.apply_H(z, y)
        return _columns(N, hp)
    raise ValueError(f"unknown operator {which!r}")


def eigenvalues(A):
    """All eigenvalues of the dense matrix A (LAPACK via numpy)."""
    return np.linalg.eigvals(np.asarray(A, dtype=np.complex128))


def summarize(lam):
    """Where a spectrum lies, in the terms of the paper's Fig. 2 discussion.

    min_abs: distance of the spectrum from the origin. disc_radius: the
    largest |lambda - 1/2|, which is at most 1/2 when the spectrum lies in
    the disc through 0 and 1 that bounds the preconditioned spectrum.
    negative_real: the fraction of eigenvalues with a negative real part.
    """
    lam = np.asarray(lam, dtype=np.complex128).ravel()
    a = np.abs(lam)
    return {
        "n": int(lam.size),
        "min_abs": float(a.min()),
        "max_abs": float(a.max()),
        "min_real": float(lam.real.min()),
        "max_real": float(lam.real.max()),
        "disc_radius": float(np.abs(lam - 0.5).max()),
        "negative_real": float(np.mean(lam.real < 0.0)),
    }


def shift_sweep(n, h, m, omega, alpha, shifts, *, precond="exact", precision="f64", f=None,
                tol=1e-8, restart=30, max_iters=5000):
    """Spectrum of the preconditioned operator and FGMRES iterations for each
    shift (beta1, beta2) in `shifts`, on one small model.

    n, h, m, omega, alpha: the grid (node counts, spacing in metres), slowness
    (one value per node, x fastest), angular frequency and damping of H
    (Eq. 2). f (optional): a right-hand side; when given, each entry also
    holds the iterations and the true relative residual of the solve to
    `tol`. Returns one dict per shift: beta, the `summarize` fields and the
    eigenvalues.
    """
    m = np.ascontiguousarray(np.asarray(m, dtype=np.float64).ravel())
    out = []
    g = helm.Grid(n, h, restart=restart, precond=precond, precision=precision,
                  max_iters=max_iters)
    try:
        g.set_model(m, omega, alpha)
        for b1, b2 in shifts:
            g.set_shift(float(b1), float(b2))
            lam = eigenvalues(dense_operator(g, "preconditioned"))
            row = {"beta": (float(b1), float(b2)), **summarize(lam), "eigenvalues": lam}
            if f is not None:
                fv = np.ascontiguousarray(np.asarray(f, dtype=np.complex128).ravel())
                u = np.empty_like(fv)
                st, its, rr = g.solve(fv, tol, u, check=False)
                row.update(status=int(st), iterations=int(its), true_rel_residual=float(rr))
            out.append(row)
    finally:
        g.close()
    return out
