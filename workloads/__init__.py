"""Seeded synthetic inputs for the heterogeneous Helmholtz solver.

This module only makes inputs: velocity models, point sources and request
streams. It holds none of the solver's arithmetic. The CPU oracle and the GPU
path both take their inputs from here and from nowhere else.

Array convention: a field on an ``n = (nx, nz)`` (2D) or ``(nx, ny, nz)`` (3D)
node grid is a numpy array of shape ``n[::-1]``. The first grid axis (x) is
the fastest-varying one, so ``a.ravel()[(iz * ny + iy) * nx + ix]`` is node
``(ix, iy, iz)``.

Stand-ins: the paper's 1D well model (Fig. 1) and its Marmousi section
(Fig. 5) have no numbers in the text. The generators below replace them with
seeded layered and smooth random media that keep the velocity range and
smoothness of those models.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy import ndimage

__all__ = [
    "layered_1d", "smooth_random", "layered_2d", "point_sources", "Workload",
    "workload", "WORKLOADS", "request_stream",
]


def layered_1d(n: int, velocities=(1500.0, 2500.0, 3500.0)) -> np.ndarray:
    """Piecewise-constant velocity on ``n`` nodes.

    The layers change at nodes ``n // 3`` and ``2 * n // 3``. An interface
    node takes the deeper layer's value.
    """
    c = np.empty(n, dtype=np.float64)
    i1, i2 = n // 3, (2 * n) // 3
    c[:i1] = velocities[0]
    c[i1:i2] = velocities[1]
    c[i2:] = velocities[2]
    return c


def _gaussian_field(shape, sigma_nodes, seed) -> np.ndarray:
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(shape)
    return ndimage.gaussian_filter(g, sigma=sigma_nodes, mode="reflect")


def smooth_random(n, h, corr_len=200.0, vmin=1500.0, vmax=4500.0, seed=0) -> np.ndarray:
    """Gaussian-smoothed white noise, rescaled affinely onto ``[vmin, vmax]``.

    ``n`` is the node count per grid axis, x first. The smoothing length is
    ``corr_len / h`` nodes.
    """
    shape = tuple(int(k) for k in n)[::-1]
    g = _gaussian_field(shape, corr_len / h, seed)
    lo, hi = g.min(), g.max()
    return vmin + (vmax - vmin) * (g - lo) / (hi - lo)


def layered_2d(n, h, n_layers=12, vmin=1500.0, vmax=4500.0, perturb=0.1,
               corr_len=200.0, seed=0) -> np.ndarray:
    """A layered 2D model with a lateral perturbation.

    The depth axis (z, the second grid axis) is split into ``n_layers`` layers
    of equal thickness. Their velocities rise linearly from ``vmin`` to
    ``vmax``. Each value is then scaled by ``1 + perturb * p``, where ``p`` is
    a smooth random field rescaled to ``[-1, 1]``. The result is clipped to
    ``[vmin, vmax]``.
    """
    nx, nz = int(n[0]), int(n[1])
    layer = np.minimum((np.arange(nz) * n_layers) // nz, n_layers - 1)
    v_layer = vmin + (vmax - vmin) * layer / max(n_layers - 1, 1)
    g = _gaussian_field((nz, nx), corr_len / h, seed)
    p = 2.0 * (g - g.min()) / (g.max() - g.min()) - 1.0
    c = v_layer[:, None] * (1.0 + perturb * p)
    return np.clip(c, vmin, vmax)


def point_sources(n, h, positions, amplitudes=None) -> np.ndarray:
    """Right-hand side with point sources ``1/h^d`` at the given nodes.

    ``positions`` is a list of node tuples ``(ix[, iy], iz)``. It returns a
    complex128 array of shape ``n[::-1]``.
    """
    n = tuple(int(k) for k in n)
    d = len(n)
    f = np.zeros(n[::-1], dtype=np.complex128)
    if amplitudes is None:
        amplitudes = [1.0] * len(positions)
    for pos, a in zip(positions, amplitudes):
        f[tuple(int(p) for p in pos)[::-1]] += a / h ** d
    return f


@dataclass
class Workload:
    """A named solve: grid, medium, frequency, shift and Krylov settings."""
    name: str
    n: tuple
    h: float
    freqs: tuple
    alpha: float
    beta: tuple
    restart: int
    tol: float
    precond: str              # "exact", "mg" or "none"
    precision: str            # "f64" or "mixed"
    sources: list
    model: str
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def unknowns(self) -> int:
        return int(np.prod(self.n))

    def velocity(self) -> np.ndarray:
        if self.model == "layered1d":
            return layered_1d(self.n[0])
        if self.model == "smooth":
            return smooth_random(self.n, self.h, seed=self.seed)
        if self.model == "layered2d":
            return layered_2d(self.n, self.h, seed=self.seed)
        raise ValueError(self.model)

    def slowness(self) -> np.ndarray:
        return 1.0 / self.velocity()

    def rhs(self, k: int | None = None) -> np.ndarray:
        """The right-hand side for source ``k`` (all sources at once if None)."""
        pos = self.sources if k is None else [self.sources[k]]
        return point_sources(self.n, self.h, pos)

    def omega(self, i: int = 0) -> float:
        return 2.0 * math.pi * self.freqs[i]


def _surface_sources(nx, count, iz=2):
    return [(int(math.floor((k + 0.5) * (nx - 1) / count + 0.5)), iz) for k in range(count)]


def workload(name: str) -> Workload:
    """The five reference workloads plus small variants used by tests.

    * ``1d_well``: 1001 nodes, h = 5 m, three layers 1500/2500/3500 m/s,
      10 Hz, alpha = 0.01, unit source 1/h at the centre node, shifted
      Laplacian (1, 0.5) applied exactly, GMRES(50), tol 1e-8.
    * ``2d_smooth``: 401 x 201 nodes, h = 10 m, smooth random medium
      (correlation 200 m) in 1500-4500 m/s, 10 Hz, source 20 m deep on the
      mid-line, V-cycle shifted Laplacian, FGMRES(30), tol 1e-8, FP64.
    * ``2d_batched``: 801 x 401 nodes, h = 7.5 m, 12-layer model with 10 %
      lateral perturbation, 64 surface sources x {5, 10, 15, 20} Hz, mixed
      precision.
    * ``3d_smooth``: 257 x 257 x 193 nodes (256 x 256 x 192 intervals),
      h = 10 m, smooth random medium, 10 Hz, 4 sources, FGMRES(20), mixed.
    """
    if name == "1d_well":
        return Workload(name, (1001,), 5.0, (10.0,), 0.01, (1.0, 0.5), 50, 1e-8,
                        "exact", "f64", [(500,)], "layered1d")
    if name == "2d_smooth":
        return Workload(name, (401, 201), 10.0, (10.0,), 0.01, (1.0, 0.5), 30, 1e-8,
                        "mg", "f64", [(200, 2)], "smooth")
    if name == "2d_smooth_small":
        return Workload(name, (101, 51), 10.0, (10.0,), 0.01, (1.0, 0.5), 30, 1e-8,
                        "mg", "f64", [(50, 2)], "smooth")
    if name == "2d_batched":
        return Workload(name, (801, 401), 7.5, (5.0, 10.0, 15.0, 20.0), 0.01, (1.0, 0.5),
                        30, 1e-8, "mg", "mixed", _surface_sources(801, 64), "layered2d")
    if name == "3d_smooth":
        return Workload(name, (257, 257, 193), 10.0, (10.0,), 0.01, (1.0, 0.5), 20, 1e-8,
                        "mg", "mixed", [(64, 64, 2), (192, 64, 2), (64, 192, 2), (192, 192, 2)],
                        "smooth")
    if name == "3d_smooth_mid":
        # the 3D medium and frequency on 129 x 129 x 97 nodes (same h and points per
        # wavelength): about 2.5 GB on the device for a 4-source batch, a size for
        # full-counter profiles
        return Workload(name, (129, 129, 97), 10.0, (10.0,), 0.01, (1.0, 0.5), 20, 1e-8,
                        "mg", "mixed", [(32, 32, 2), (96, 32, 2), (32, 96, 2), (96, 96, 2)],
                        "smooth")
    if name == "3d_smooth_small":
        return Workload(name, (33, 33, 25), 10.0, (10.0,), 0.01, (1.0, 0.5), 20, 1e-8,
                        "mg", "mixed", [(16, 16, 2)], "smooth")
    raise KeyError(name)


WORKLOADS = ("1d_well", "2d_smooth", "2d_batched", "3d_smooth")

SERVING_GRIDS = ((257, 129), (513, 257), (1025, 513), (1601, 801))


def request_stream(count: int, rate_hz: float = 200.0, seed: int = 0, h: float = 10.0,
                   grids=SERVING_GRIDS, ppw: float = 10.0, c_min: float = 1500.0):
    """A Poisson stream of 2D solve requests.

    Each request draws a grid uniformly from ``grids``, one to eight sources
    at depth node 2 with uniform random x nodes, and its own model seed. The
    frequency gives ``ppw`` points per wavelength at ``c_min``. Returns a list
    of dicts with ``t_arrival`` in seconds.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    freq = c_min / (ppw * h)
    for i in range(count):
        t += rng.exponential(1.0 / rate_hz)
        g = grids[int(rng.integers(len(grids)))]
        ns = int(rng.integers(1, 9))
        xs = rng.integers(1, g[0] - 1, size=ns)
        out.append({
            "id": i, "t_arrival": t, "n": tuple(g), "h": h, "freq": freq,
            "sources": [(int(x), 2) for x in xs], "model_seed": int(rng.integers(1 << 31)),
        })
    return out
