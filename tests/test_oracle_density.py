"""Pins of the variable-density oracle operator (Eq. 1): reductions to the
constant-density operator of Eq. 2, symmetry of the flux form, and the
second-order convergence of a manufactured solution."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import closed_form as cf
from oracle import density
from oracle import operator as op


def _rand(n, seed, lo, hi):
    return np.random.default_rng(seed).uniform(lo, hi, size=tuple(n)[::-1])


@pytest.mark.parametrize("n", [(9,), (7, 6), (4, 3, 5)])
def test_unit_rho_is_the_constant_density_operator(n):
    h, om, al = 10.0, 2 * np.pi * 10.0, 0.01
    m = 1.0 / _rand(n, 1, 1500.0, 4500.0)
    A = density.assemble_H_rho(n, h, m, np.ones(int(np.prod(n))), om, al).toarray()
    B = op.assemble_H(n, h, m, om, al).toarray()
    assert np.abs(A - B).max() <= 1e-14 * np.abs(B).max()


@pytest.mark.parametrize("n", [(9,), (7, 6), (4, 3, 5)])
def test_constant_rho_scales_the_operator(n):
    """-div(rho0 grad u) - k^2 (1 - j alpha) u = rho0 [-Lap u - (k^2 / rho0)
    (1 - j alpha) u], and the outgoing wavenumber kappa / sqrt(rho0) is that of
    the slowness m / sqrt(rho0): H_rho(rho0, m) = rho0 H(m / sqrt(rho0))."""
    h, om, al, r0 = 10.0, 2 * np.pi * 10.0, 0.01, 2.7
    m = 1.0 / _rand(n, 2, 1500.0, 4500.0)
    A = density.assemble_H_rho(n, h, m, np.full(int(np.prod(n)), r0), om, al).toarray()
    B = r0 * op.assemble_H(n, h, m / np.sqrt(r0), om, al).toarray()
    assert np.abs(A - B).max() <= 1e-13 * np.abs(B).max()


@pytest.mark.parametrize("n", [(9,), (7, 6), (4, 3, 5)])
def test_flux_form_is_symmetric(n):
    """Face coefficients shared by the two rows of a face: D H is complex
    symmetric (D: 1/2 per boundary face), for any positive rho."""
    h, om, al = 10.0, 2 * np.pi * 10.0, 0.01
    m = 1.0 / _rand(n, 3, 1500.0, 4500.0)
    rho = _rand(n, 4, 0.5, 3.0)
    A = density.assemble_H_rho(n, h, m, rho, om, al).toarray()
    DA = op.boundary_weights(n)[:, None] * A
    assert np.abs(DA - DA.T).max() <= 1e-15 * np.abs(DA).max()
    # and it is not symmetric without the face averaging (a check that the
    # test can fail): node-value coefficients break it
    Bad = A.copy()
    i = int(np.prod(n)) // 2
    Bad[i, i + 1] *= 1.1
    DB = op.boundary_weights(n)[:, None] * Bad
    assert np.abs(DB - DB.T).max() > 1e-6 * np.abs(DA).max()


def _rho(X, L):
    """rho = 1.5 + 0.5 prod_a cos(pi x_a / L_a): zero normal derivative on the
    faces of the box, where the mirrored ghost face is second order."""
    p = np.ones_like(X[0])
    for a in range(len(L)):
        p = p * np.cos(np.pi * X[a] / L[a])
    return 1.5 + 0.5 * p


def _drho(X, L, a):
    p = -0.5 * (np.pi / L[a]) * np.sin(np.pi * X[a] / L[a])
    for b in range(len(L)):
        if b != a:
            p = p * np.cos(np.pi * X[b] / L[b])
    return p


def _manufactured_rhs(ms, n, h):
    """f = -div(rho grad u*) - k^2 (1 - j alpha) u* at every node, plus
    2 rho_face g / h on each boundary face, g = dn u* + j (kappa/sqrt(rho)) u*."""
    X = ms._grid(n)
    L = ms.L
    u = ms.u(n)
    m = ms.slowness(n)
    rho = _rho(X, L)
    re = np.ones_like(X[0])
    for a in range(ms.d):
        re = re * np.cos(ms.k[a] * X[a] + ms.t[a])
    lap = -np.sum(ms.k ** 2) * re                 # the imaginary part is multilinear
    div = rho * lap
    for a in range(ms.d):
        div = div + _drho(X, L, a) * ms._du(X, a)
    f = -div - ms.omega ** 2 * m ** 2 * (1.0 - 1j * ms.alpha) * u
    kap = ms.omega * m * np.sqrt(1.0 - 1j * ms.alpha) / np.sqrt(rho)
    for a in range(ms.d):
        ax = ms.d - 1 - a
        du = ms._du(X, a)
        lo = X[a] == 0.0
        hi = np.isclose(X[a], L[a])
        # face coefficient between the boundary node and its inner neighbour
        b_lo = 0.5 * (rho + np.roll(rho, -1, axis=ax))
        b_hi = 0.5 * (rho + np.roll(rho, 1, axis=ax))
        f = f + np.where(lo, 2.0 * b_lo * (-du + 1j * kap * u) / h, 0.0)
        f = f + np.where(hi, 2.0 * b_hi * (du + 1j * kap * u) / h, 0.0)
    return f, rho, m


def test_manufactured_variable_density_2d_second_order():
    om, al = 2 * np.pi * 8.0, 0.01
    lengths = (2000.0, 1000.0)
    errs = []
    for k in (8, 16, 32, 64):
        n = tuple(int(round(L / lengths[1] * k)) + 1 for L in lengths)
        h = lengths[1] / k
        ms = cf.Manufactured(lengths, om, al)
        f, rho, m = _manufactured_rhs(ms, n, h)
        H = density.assemble_H_rho(n, h, m, rho, om, al)
        u = spla.spsolve(H.tocsc(), f.ravel())
        errs.append(np.abs(u - ms.u(n).ravel()).max())
    e = np.array(errs)
    order = np.log2(e[:-1] / e[1:])
    assert np.all(order[-2:] > 1.8) and np.all(order[-2:] < 2.3), order


def test_rejects_bad_coefficients():
    with pytest.raises(ValueError):
        density.assemble_H_rho((5,), 1.0, np.ones(5), np.zeros(5), 1.0, 0.0)
    with pytest.raises(ValueError):
        density.assemble_H_rho((5,), 1.0, np.ones(4), np.ones(5), 1.0, 0.0)


# ---------------------------------------------------------------- the shifted Laplacian with rho

@pytest.mark.parametrize("n", [(9,), (7, 6), (4, 3, 5)])
def test_unit_rho_M_is_the_constant_density_M(n):
    """Eq. 6 with rho = 1: the shifted Laplacian of the constant-density oracle."""
    h, om, al, b = 10.0, 2 * np.pi * 10.0, 0.01, (1.0, 0.5)
    m = 1.0 / _rand(n, 5, 1500.0, 4500.0)
    A = density.assemble_M_rho(n, h, m, np.ones(int(np.prod(n))), om, al, *b).toarray()
    B = op.assemble_M(n, h, m, om, al, *b).toarray()
    assert np.abs(A - B).max() <= 1e-14 * np.abs(B).max()


@pytest.mark.parametrize("n", [(9,), (7, 6), (4, 3, 5)])
def test_H_minus_M_is_diagonal_with_rho(n):
    """M_rho keeps the divergence and boundary rows of H_rho, so H_rho - M_rho is
    -omega^2 m^2 [(1 - j alpha) - (beta1 - j beta2)] on the diagonal and 0 elsewhere."""
    h, om, al, b = 10.0, 2 * np.pi * 10.0, 0.01, (1.0, 0.5)
    m = 1.0 / _rand(n, 6, 1500.0, 4500.0)
    rho = _rand(n, 7, 0.5, 3.0)
    D = (density.assemble_H_rho(n, h, m, rho, om, al)
         - density.assemble_M_rho(n, h, m, rho, om, al, *b)).toarray()
    want = -om ** 2 * m.ravel() ** 2 * ((1 - 1j * al) - (b[0] - 1j * b[1]))
    assert np.abs(D - np.diag(want)).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("n", [(9,), (7, 6)])
def test_constant_rho_scales_M(n):
    h, om, al, r0, b = 10.0, 2 * np.pi * 10.0, 0.01, 0.6, (1.0, 0.5)
    m = 1.0 / _rand(n, 8, 1500.0, 4500.0)
    A = density.assemble_M_rho(n, h, m, np.full(int(np.prod(n)), r0), om, al, *b).toarray()
    B = r0 * op.assemble_M(n, h, m / np.sqrt(r0), om, al, *b).toarray()
    assert np.abs(A - B).max() <= 1e-13 * np.abs(B).max()


def test_unit_rho_levels_are_the_constant_density_levels():
    from oracle import multigrid as mg
    n, h, om, al, b = (33, 17), 10.0, 2 * np.pi * 10.0, 0.01, (1.0, 0.5)
    m = 1.0 / _rand(n, 9, 1500.0, 4500.0)
    La = density.build_levels_rho(n, h, m, np.ones(m.shape), om, al, *b, coarse_max=100)
    Lb = mg.build_levels(n, h, m, om, al, *b, coarse_max=100)
    assert [L.n for L in La] == [L.n for L in Lb] and len(La) == 3
    for A, B in zip(La, Lb):
        assert abs(A.h - B.h) < 1e-12
        assert np.abs((A.M - B.M).toarray()).max() <= 1e-14 * np.abs(B.M.toarray()).max()


def test_rho_levels_inject_rho():
    """Each coarse level's M_rho is the operator of the injected rho (a hierarchy
    that kept rho = 1 below the fine level, or shifted the injection by one
    node, fails this)."""
    n, h, om, al, b = (17, 9), 10.0, 2 * np.pi * 10.0, 0.01, (1.0, 0.5)
    m = 1.0 / _rand(n, 10, 1500.0, 4500.0)
    rho = _rand(n, 11, 0.5, 3.0)
    L = density.assemble_M_rho
    levels = density.build_levels_rho(n, h, m, rho, om, al, *b, coarse_max=50)
    assert len(levels) == 2
    want = L((9, 5), 2 * h, m[::2, ::2], rho[::2, ::2], om, al, *b).toarray()
    assert np.abs(levels[1].M.toarray() - want).max() <= 1e-14 * np.abs(want).max()


def test_vcycle_with_rho_contracts():
    """V(1,1) on M_rho with a smooth rho in [0.5, 2.5]: the error propagator
    I - B M_rho (B the V-cycle) has spectral radius below 0.65, measured by
    power iteration (0.58 here; the same grid with rho = 1 gives 0.65). A
    hierarchy whose coarse levels ignore rho diverges (radius > 1)."""
    from oracle import multigrid as mg
    n, h, om, al, b = (65, 33), 10.0, 2 * np.pi * 10.0, 0.01, (1.0, 0.5)
    rng = np.random.default_rng(12)
    m = 1.0 / rng.uniform(1500.0, 4500.0, size=n[::-1])
    y, x = np.meshgrid(np.arange(n[1]), np.arange(n[0]), indexing="ij")
    rho = 1.5 + np.sin(2 * np.pi * x / 64.0) * np.cos(np.pi * y / 32.0)
    levels = density.build_levels_rho(n, h, m, rho, om, al, *b, coarse_max=300)
    assert len(levels) == 3
    M = levels[0].M

    def radius(lv):
        e = np.random.default_rng(13).standard_normal(M.shape[0]) + 0j
        rate = 0.0
        for _ in range(30):
            e2 = e - mg.vcycle(lv, M @ e, 1, 1, 0.8)
            rate = np.linalg.norm(e2) / np.linalg.norm(e)
            e = e2 / np.linalg.norm(e2)
        return rate

    assert radius(levels) < 0.65
    wrong = [levels[0]] + mg.build_levels(n, h, m, om, al, *b, coarse_max=300)[1:]
    assert radius(wrong) > 1.0
