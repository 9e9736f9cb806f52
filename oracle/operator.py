"""Sparse assembly of the Helmholtz operator and of the shifted Laplacian.

Continuous model (Eq. 2): -Lap u - omega^2 m^2 (1 - j alpha) u = f, with
m = 1/c the slowness, and a first-order absorbing boundary (Summary and
Eq. 1). Matrix form H u = f (Eq. 3).

Readings of what the paper leaves open (all stated in the design notes):

* Second-order finite differences on a node-centred grid. Every node,
  boundary nodes included, is an unknown. The stencil has 3 points in 1D,
  5 in 2D and 7 in 3D, with the coefficient taken at the node.
* The absorbing condition is dn u + j kappa u = 0, with
  kappa = omega m sqrt(1 - j alpha) (principal root, Im kappa < 0). This is
  the outgoing condition for the e^{-j kappa |x|} Green's function that goes
  with the sign of the damping term in Eq. 2.
* That condition is imposed by a centred ghost node: u_ghost = u_in -
  2 j h kappa u_b. On a boundary row this doubles the inward neighbour and
  adds 2 j kappa / h to the diagonal, once for each face the node lies on.
* The preconditioner of Eq. 6 is written as M = -Lap - (beta1 - j beta2)
  omega^2 m^2. It has the same Laplacian and boundary rows as H. The
  paper's P = -Lap + beta k^2 with beta = b1 + j b2 is M with
  (beta1, beta2) = (-b1, b2).

Index convention: node (i0, i1, i2) with i0 fastest; flat index
``(i2 * n1 + i1) * n0 + i0``. Arrays have shape ``n[::-1]``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = ["kappa", "laplacian_bc", "assemble_H", "assemble_M", "assemble_shifted",
           "boundary_weights", "sigma_H", "sigma_M"]


def kappa(omega: float, m: np.ndarray, alpha: float) -> np.ndarray:
    """Damped wavenumber kappa = omega m sqrt(1 - j alpha), principal root."""
    return omega * np.asarray(m, dtype=np.float64) * np.sqrt(1.0 - 1j * alpha)


def sigma_H(omega, m, alpha):
    """Zero-order coefficient of H: omega^2 m^2 (1 - j alpha) (Eq. 2)."""
    return omega ** 2 * np.asarray(m, dtype=np.float64) ** 2 * (1.0 - 1j * alpha)


def sigma_M(omega, m, beta1, beta2):
    """Zero-order coefficient of M: (beta1 - j beta2) omega^2 m^2 (Eq. 6)."""
    return (beta1 - 1j * beta2) * omega ** 2 * np.asarray(m, dtype=np.float64) ** 2


def laplacian_bc(n, h, kb) -> sp.csr_matrix:
    """-Lap with ghost-node absorbing rows, as a CSR matrix.

    ``n``: node counts per axis (axis 0 fastest), each at least 2.
    ``kb``: complex kappa at every node (shape ``n[::-1]``), used on the
    boundary rows only.
    """
    n = tuple(int(k) for k in n)
    if any(k < 2 for k in n):
        raise ValueError("every axis needs at least 2 nodes")
    shape = n[::-1]
    N = int(np.prod(n))
    idx = np.arange(N).reshape(shape)
    kb = np.broadcast_to(np.asarray(kb, dtype=np.complex128), shape)
    diag = np.zeros(shape, dtype=np.complex128)
    rows, cols, vals = [], [], []
    inv_h2 = 1.0 / (h * h)
    for a in range(len(n)):
        ax = len(n) - 1 - a                       # numpy axis of grid axis a
        coord = np.arange(n[a]).reshape([-1 if k == ax else 1 for k in range(len(n))])
        coord = np.broadcast_to(coord, shape)
        lower_bnd = coord == 0
        upper_bnd = coord == n[a] - 1
        diag += 2.0 * inv_h2
        # a node on a face gets 2 j kappa / h from the ghost node there
        diag += np.where(lower_bnd, 2j * kb / h, 0.0)
        diag += np.where(upper_bnd, 2j * kb / h, 0.0)
        # neighbour below (i_a - 1): exists unless on the lower face; its
        # weight doubles when the node above is a ghost (upper face)
        has_lo = ~lower_bnd
        w_lo = np.where(upper_bnd, -2.0 * inv_h2, -1.0 * inv_h2)
        rows.append(idx[has_lo])
        cols.append(np.roll(idx, 1, axis=ax)[has_lo])
        vals.append(w_lo[has_lo].astype(np.complex128))
        has_hi = ~upper_bnd
        w_hi = np.where(lower_bnd, -2.0 * inv_h2, -1.0 * inv_h2)
        rows.append(idx[has_hi])
        cols.append(np.roll(idx, -1, axis=ax)[has_hi])
        vals.append(w_hi[has_hi].astype(np.complex128))
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    return A.tocsr()


def assemble_shifted(n, h, m, omega, alpha, shift) -> sp.csr_matrix:
    """-Lap_bc - diag(shift * omega^2 m^2), boundary rows with damped kappa."""
    m = np.asarray(m, dtype=np.float64).reshape(tuple(int(k) for k in n)[::-1])
    L = laplacian_bc(n, h, kappa(omega, m, alpha))
    s = shift * omega ** 2 * m.ravel() ** 2
    return (L - sp.diags(s)).tocsr()


def assemble_H(n, h, m, omega, alpha) -> sp.csr_matrix:
    """The Helmholtz matrix H of Eq. 3 (shift factor 1 - j alpha)."""
    return assemble_shifted(n, h, m, omega, alpha, 1.0 - 1j * alpha)


def assemble_M(n, h, m, omega, alpha, beta1, beta2) -> sp.csr_matrix:
    """The shifted Laplacian of Eq. 6 in the (beta1 - j beta2) convention.

    ``alpha`` only enters through kappa on the boundary rows, so that H - M
    is diagonal.
    """
    return assemble_shifted(n, h, m, omega, alpha, beta1 - 1j * beta2)


def boundary_weights(n) -> np.ndarray:
    """D: 1/2 per face a node lies on. D H is complex symmetric."""
    n = tuple(int(k) for k in n)
    shape = n[::-1]
    w = np.ones(shape)
    for a in range(len(n)):
        ax = len(n) - 1 - a
        coord = np.broadcast_to(
            np.arange(n[a]).reshape([-1 if k == ax else 1 for k in range(len(n))]), shape)
        w = w * np.where((coord == 0) | (coord == n[a] - 1), 0.5, 1.0)
    return w.ravel()
