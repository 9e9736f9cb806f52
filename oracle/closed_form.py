"""Closed forms that pin the discretisation of Eq. 2 with absorbing boundaries.

* ``discrete_1d``: the exact solution of the 3-point scheme for constant
  kappa and one point source. Away from the source and the two ends, the
  rows are the recurrence u_{i+1} + u_{i-1} = (2 - kappa^2 h^2) u_i, whose
  solutions are a z^i + b z^-i with z + 1/z = 2 - kappa^2 h^2. Four
  conditions fix the four coefficients: continuity at the source, the
  source row and the two boundary rows.
* ``green_1d``: the continuous outgoing Green's function
  G(x) = exp(-j kappa |x - xs|) / (2 j kappa). It solves
  -G'' - kappa^2 G = delta(x - xs) and meets dn G + j kappa G = 0 exactly,
  so the discrete solution must converge to it at second order.
* ``manufactured``: a smooth complex field u*, the source f = H u* computed
  by hand-derived derivatives, and the boundary data
  g = dn u* + j kappa u*, for a second-order convergence check in 2D and 3D.
"""
from __future__ import annotations

import numpy as np

__all__ = ["discrete_1d", "green_1d", "Manufactured"]


def discrete_1d(n: int, h: float, kappa: complex, s: int, fs: complex) -> np.ndarray:
    """Exact nodal solution of the 1D scheme with a source ``fs`` at node s."""
    if not 1 <= s <= n - 2:
        raise ValueError("source must be an interior node")
    k2h2 = kappa * kappa * h * h
    t = 2.0 - k2h2
    disc = np.sqrt(t * t - 4.0 + 0j)
    z = (t + disc) / 2.0
    if abs(z) > 1.0:
        z = 1.0 / z
    r = n - 1 - s
    # left: u_i = a z^i + b z^-i (0 <= i <= s);
    # right: u_i = c z^(i-s) + d z^-(i-s) (s <= i <= n-1)
    A = np.zeros((4, 4), dtype=np.complex128)
    rhs = np.zeros(4, dtype=np.complex128)
    # continuity at s
    A[0] = [z ** s, z ** (-s), -1.0, -1.0]
    # source row: (2 u_s - u_{s-1} - u_{s+1}) / h^2 - kappa^2 u_s = fs
    A[1] = [-z ** (s - 1) / h ** 2, -z ** (-(s - 1)) / h ** 2,
            (2.0 - k2h2) / h ** 2 - z / h ** 2, (2.0 - k2h2) / h ** 2 - 1.0 / (z * h ** 2)]
    rhs[1] = fs
    # left end: (2 u_0 - 2 u_1) / h^2 + (2 j kappa / h) u_0 - kappa^2 u_0 = 0
    d0 = 2.0 / h ** 2 + 2j * kappa / h - kappa * kappa
    A[2] = [d0 - 2.0 * z / h ** 2, d0 - 2.0 / (z * h ** 2), 0.0, 0.0]
    # right end, same form at node n-1 with inward neighbour n-2
    A[3] = [0.0, 0.0, d0 * z ** r - 2.0 * z ** (r - 1) / h ** 2,
            d0 * z ** (-r) - 2.0 * z ** (-(r - 1)) / h ** 2]
    a, b, c, d = np.linalg.solve(A, rhs)
    i = np.arange(n)
    u = np.where(i <= s, a * z ** i.astype(float) + b * z ** (-i.astype(float)),
                 c * z ** (i - s).astype(float) + d * z ** (-(i - s).astype(float)))
    return u


def green_1d(x, xs, kappa):
    """Outgoing Green's function of -d2/dx2 - kappa^2."""
    return np.exp(-1j * kappa * np.abs(np.asarray(x) - xs)) / (2j * kappa)


class Manufactured:
    """u*(x) = prod_a cos(k_a x_a + t_a) + j prod_a (x_a / L_a).

    The slowness is m(x) = 1 / (2000 + 600 prod_a cos(pi x_a / L_a)).
    Derivatives are written by hand: the imaginary part is multilinear, so
    its Laplacian vanishes.
    """

    def __init__(self, lengths, omega, alpha):
        self.L = np.asarray(lengths, dtype=np.float64)
        self.d = len(lengths)
        self.k = np.array([1.3, 2.1, 0.9][:self.d]) * np.pi / self.L
        self.t = np.array([0.3, -0.7, 1.1][:self.d])
        self.omega = omega
        self.alpha = alpha

    def _grid(self, n):
        axes = [np.linspace(0.0, self.L[a], int(n[a])) for a in range(self.d)]
        mesh = np.meshgrid(*axes[::-1], indexing="ij")   # arrays of shape n[::-1]
        return mesh[::-1]                               # coordinate a -> x_a

    def slowness(self, n):
        X = self._grid(n)
        p = np.ones_like(X[0])
        for a in range(self.d):
            p = p * np.cos(np.pi * X[a] / self.L[a])
        return 1.0 / (2000.0 + 600.0 * p)

    def u(self, n):
        X = self._grid(n)
        re = np.ones_like(X[0])
        im = np.ones_like(X[0])
        for a in range(self.d):
            re = re * np.cos(self.k[a] * X[a] + self.t[a])
            im = im * X[a] / self.L[a]
        return re + 1j * im

    def _du(self, X, a):
        """Partial derivative of u* along axis a."""
        re = -self.k[a] * np.sin(self.k[a] * X[a] + self.t[a])
        im = np.full_like(X[0], 1.0 / self.L[a])
        for b in range(self.d):
            if b != a:
                re = re * np.cos(self.k[b] * X[b] + self.t[b])
                im = im * X[b] / self.L[b]
        return re + 1j * im

    def rhs(self, n):
        """f = H u* at every node plus 2 g / h on each boundary face."""
        X = self._grid(n)
        h = self.L[0] / (int(n[0]) - 1)
        m = self.slowness(n)
        re = np.ones_like(X[0])
        for a in range(self.d):
            re = re * np.cos(self.k[a] * X[a] + self.t[a])
        lap = -np.sum(self.k ** 2) * re
        u = self.u(n)
        f = -lap - self.omega ** 2 * m ** 2 * (1.0 - 1j * self.alpha) * u
        kap = self.omega * m * np.sqrt(1.0 - 1j * self.alpha)
        for a in range(self.d):
            du = self._du(X, a)
            lo = X[a] == 0.0
            hi = np.isclose(X[a], self.L[a])
            g_lo = -du + 1j * kap * u
            g_hi = du + 1j * kap * u
            f = f + np.where(lo, 2.0 * g_lo / h, 0.0) + np.where(hi, 2.0 * g_hi / h, 0.0)
        return f
