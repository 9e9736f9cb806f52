"""Variable-density Helmholtz operator (Eq. 1) for the oracle.

TEST INFRASTRUCTURE: only the tests may import this module; no product
code calls it.

Eq. 1 as printed: -div(rho grad u) - k^2 (1 - j alpha) u = f, with
k = omega m. For constant rho = 1 it reduces to Eq. 2. The readings below
are stated in the design notes.

* rho is the coefficient inside the divergence, as printed. For the
  acoustic pressure equation a caller passes 1/density.
* Conservative second-order differences on the node-centred grid. On the
  face between two neighbouring nodes the coefficient is the arithmetic
  mean of their values, so the row for node p along one axis reads
  [rho_(p-1/2) (u_p - u_(p-1)) + rho_(p+1/2) (u_p - u_(p+1))] / h^2.
* Absorbing boundary. The outgoing wave of -div(rho grad u) - kappa^2 u = 0
  with rho locally constant has wavenumber kappa / sqrt(rho). So the
  first-order condition is dn u + j (kappa / sqrt(rho)) u = 0, with
  kappa = omega m sqrt(1 - j alpha) (principal root), taken at the boundary
  node.
* It is imposed by a ghost node at distance h outside the face, as in the
  constant-density operator: u_ghost = u_in - 2 j h (kappa / sqrt(rho)) u_b.
  The ghost face takes the coefficient of the inner face (mirror), so a
  boundary row along that axis is
  rho_in_face [2 u_b - 2 u_in + 2 j h (kappa / sqrt(rho_b)) u_b] / h^2.
  A node on several faces gets one such term per face.

These readings give:
* rho = 1 is the operator of Eq. 2;
* rho = rho0 (constant) is rho0 times the Eq. 2 operator of slowness
  m / sqrt(rho0);
* D H is complex symmetric (D: 1/2 per face a node lies on).
The tests check these.

Index convention as the constant-density oracle: node (i0, i1, i2) with i0
fastest; flat index (i2 * n1 + i1) * n0 + i0; arrays have shape n[::-1].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = ["assemble_shifted_rho", "assemble_H_rho", "assemble_M_rho", "build_levels_rho"]


def assemble_shifted_rho(n, h, m, rho, omega, alpha, shift) -> sp.csr_matrix:
    """-div(rho grad) with the absorbing rows above, minus shift * omega^2 m^2,
    as a CSR matrix assembled node by node.

    n: node counts per axis (axis 0 fastest, each >= 2); h: spacing;
    m: slowness and rho: the coefficient of Eq. 1, one value per node (shape
    n[::-1] or flat); omega: angular frequency; alpha: damping, which enters
    the boundary rows through kappa; shift: the complex factor of the
    zero-order term (1 - j alpha for H, beta1 - j beta2 for M).
    """
    n = tuple(int(k) for k in n)
    if any(k < 2 for k in n):
        raise ValueError("every axis needs at least 2 nodes")
    d = len(n)
    N = int(np.prod(n))
    m = np.asarray(m, dtype=np.float64).ravel()
    rho = np.asarray(rho, dtype=np.float64).ravel()
    if m.size != N or rho.size != N:
        raise ValueError("m and rho need one value per node")
    if np.any(rho <= 0.0):
        raise ValueError("rho must be positive")
    stride = [int(np.prod(n[:a])) for a in range(d)]   # 1, n0, n0 n1
    kap = omega * m * np.sqrt(1.0 - 1j * alpha)
    ih2 = 1.0 / (h * h)
    A = sp.lil_matrix((N, N), dtype=np.complex128)
    for p in range(N):
        idx = [(p // stride[a]) % n[a] for a in range(d)]
        diag = -shift * omega ** 2 * m[p] ** 2
        for a in range(d):
            i = idx[a]
            lo = p - stride[a] if i > 0 else None
            hi = p + stride[a] if i < n[a] - 1 else None
            if lo is not None and hi is not None:
                b_lo = 0.5 * (rho[p] + rho[lo])
                b_hi = 0.5 * (rho[p] + rho[hi])
                diag += (b_lo + b_hi) * ih2
                A[p, lo] += -b_lo * ih2
                A[p, hi] += -b_hi * ih2
            else:
                inner = hi if lo is None else lo
                b_in = 0.5 * (rho[p] + rho[inner])
                kb = kap[p] / np.sqrt(rho[p])
                diag += b_in * (2.0 + 2j * h * kb) * ih2
                A[p, inner] += -2.0 * b_in * ih2
        A[p, p] += diag
    return A.tocsr()


def assemble_H_rho(n, h, m, rho, omega, alpha) -> sp.csr_matrix:
    """H of Eq. 1 (variable rho): the zero-order factor is 1 - j alpha."""
    return assemble_shifted_rho(n, h, m, rho, omega, alpha, 1.0 - 1j * alpha)


def assemble_M_rho(n, h, m, rho, omega, alpha, beta1, beta2) -> sp.csr_matrix:
    """The shifted Laplacian of Eq. 6 for the operator of Eq. 1: the same
    -div(rho grad) and boundary rows as H_rho, zero-order factor
    beta1 - j beta2 (so that H_rho - M_rho is diagonal, as without rho)."""
    return assemble_shifted_rho(n, h, m, rho, omega, alpha, beta1 - 1j * beta2)


def build_levels_rho(n, h, m, rho, omega, alpha, beta1, beta2, coarse_max=1500, max_levels=32):
    """Multigrid levels of M_rho: the coarsening rule of the constant-density
    hierarchy, with both the slowness and rho injected (coarse node =
    coincident fine node) and M_rho rediscretised on every level. The result
    feeds multigrid.vcycle unchanged."""
    from .multigrid import Level, can_coarsen
    n = tuple(int(k) for k in n)
    m = np.asarray(m, dtype=np.float64).reshape(n[::-1])
    rho = np.asarray(rho, dtype=np.float64).reshape(n[::-1])
    levels = []
    while True:
        levels.append(Level(n, h, m, assemble_M_rho(n, h, m, rho, omega, alpha, beta1, beta2)))
        if int(np.prod(n)) <= coarse_max or not can_coarsen(n) or len(levels) >= max_levels:
            break
        sl = tuple(slice(None, None, 2) for _ in n)
        m, rho = m[sl], rho[sl]
        n = tuple((k + 1) // 2 for k in n)
        h = 2.0 * h
    return levels
