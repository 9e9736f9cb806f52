"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than its own formulas:
closed forms, convergence under refinement, an independent Kronecker-sum
construction, dense brute force, invariants, and the paper's spectral
claim (Example section, Fig. 2).
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import closed_form as cf
from oracle import direct, gmres
from oracle import multigrid as mg
from oracle import operator as op

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- 1D closed forms (K1, K2)

@pytest.mark.parametrize("n,s,c", [(101, 40, 2000.0), (64, 10, 1500.0), (257, 200, 3500.0)])
def test_discrete_1d_closed_form(n, s, c):
    """The sparse LU solution equals the exact solution of the recurrence."""
    h, om, al = 5.0, 2 * np.pi * 10.0, 0.01
    m = np.full(n, 1.0 / c)
    f = np.zeros(n, complex)
    f[s] = 1.0 / h
    u = direct.lu_solve((n,), h, m, om, al, f)
    ue = cf.discrete_1d(n, h, op.kappa(om, m, al)[0], s, 1.0 / h)
    assert np.abs(u - ue).max() / np.abs(ue).max() < 1e-12


def test_green_function_second_order():
    """Point-source solutions converge to exp(-j k|x-xs|)/(2jk) at O(h^2)."""
    om, al, L = 2 * np.pi * 10.0, 0.01, 2000.0
    errs = []
    for n in (201, 401, 801, 1601):
        h = L / (n - 1)
        m = np.full(n, 1.0 / 2000.0)
        s = (n - 1) // 2
        f = np.zeros(n, complex)
        f[s] = 1.0 / h
        u = direct.lu_solve((n,), h, m, om, al, f)
        G = cf.green_1d(np.arange(n) * h, s * h, op.kappa(om, m, al)[0])
        errs.append(np.abs(u - G).max() / np.abs(G).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 3.8) & (ratios < 4.2)), ratios


def test_green_function_rejects_wrong_boundary_sign():
    """With the opposite sign in the boundary term the error does not shrink.

    This is what makes the outgoing reading of the absorbing condition
    checkable: the incoming version reflects and stays O(1) away from G.
    """
    om, al, L, n = 2 * np.pi * 10.0, 0.01, 2000.0, 801
    h = L / (n - 1)
    m = np.full(n, 1.0 / 2000.0)
    kap = op.kappa(om, m, al)
    s = (n - 1) // 2
    f = np.zeros(n, complex)
    f[s] = 1.0 / h
    bad = op.laplacian_bc((n,), h, -np.conj(kap)) - sp.diags(op.sigma_H(om, m, al))
    u = spla.spsolve(bad.tocsc(), f)
    G = cf.green_1d(np.arange(n) * h, s * h, kap[0])
    assert np.abs(u - G).max() / np.abs(G).max() > 0.1


# ---------------------------------------------------------------- manufactured solution (K3)

def _manufactured_errors(d, ks):
    om, al = 2 * np.pi * 8.0, 0.01
    lengths = (2000.0, 1000.0, 1500.0)[:d]
    errs = []
    for k in ks:
        n = tuple(int(round(L / lengths[1] * k)) + 1 for L in lengths)
        h = lengths[1] / k
        ms = cf.Manufactured(lengths, om, al)
        H = op.assemble_H(n, h, ms.slowness(n), om, al)
        u = spla.spsolve(H.tocsc(), ms.rhs(n).ravel())
        errs.append(np.abs(u - ms.u(n).ravel()).max())
    return np.array(errs)


def test_manufactured_2d_second_order():
    e = _manufactured_errors(2, (16, 32, 64, 128))
    order = np.log2(e[:-1] / e[1:])
    assert np.all(order[-2:] > 1.8) and np.all(order[-2:] < 2.3), order


def test_manufactured_3d_second_order():
    e = _manufactured_errors(3, (6, 12, 24))
    order = np.log2(e[:-1] / e[1:])
    assert order[-1] > 1.7 and order[-1] < 2.4, order


# ---------------------------------------------------------------- brute force (K4)

def _k1d(n, h, kap):
    """1D -d2/dx2 with absorbing ends, written row by row."""
    K = np.zeros((n, n), complex)
    for i in range(n):
        K[i, i] = 2.0 / h ** 2
        if i == 0:
            K[i, i] += 2j * kap / h
            K[i, 1] = -2.0 / h ** 2
        elif i == n - 1:
            K[i, i] += 2j * kap / h
            K[i, n - 2] = -2.0 / h ** 2
        else:
            K[i, i - 1] = K[i, i + 1] = -1.0 / h ** 2
    return K


@pytest.mark.parametrize("n", [(64,), (8, 8), (4, 4, 4), (5, 3), (3, 4, 2)])
def test_kronecker_sum_and_dense_solve(n):
    """Constant medium: H equals a Kronecker sum of 1D operators, and splu
    equals a dense solve."""
    h, om, al, c = 7.0, 2 * np.pi * 12.0, 0.05, 1800.0
    m = np.full(n[::-1], 1.0 / c)
    kap = op.kappa(om, 1.0 / c, al)
    H = op.assemble_H(n, h, m, om, al).toarray()
    N = int(np.prod(n))
    K = np.zeros((N, N), complex)
    for a in range(len(n)):
        left = np.eye(int(np.prod(n[a + 1:])))
        right = np.eye(int(np.prod(n[:a])))
        K += np.kron(left, np.kron(_k1d(n[a], h, kap), right))
    K -= np.eye(N) * om ** 2 / c ** 2 * (1 - 1j * al)
    assert np.abs(H - K).max() <= 1e-12 * np.abs(K).max()
    rng = np.random.default_rng(1)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    u1 = np.linalg.solve(K, f)
    u2 = spla.splu(sp.csc_matrix(H)).solve(f)
    assert np.linalg.norm(u1 - u2) <= 1e-12 * np.linalg.norm(u1)


# ---------------------------------------------------------------- invariants (K5)

def test_H_minus_M_is_diagonal_and_DH_symmetric():
    rng = np.random.default_rng(3)
    n, h, om, al, b1, b2 = (9, 7), 10.0, 2 * np.pi * 10, 0.01, 1.0, 0.5
    m = 1.0 / rng.uniform(1500, 4500, size=n[::-1])
    H = op.assemble_H(n, h, m, om, al)
    M = op.assemble_M(n, h, m, om, al, b1, b2)
    Dm = (H - M).toarray()
    expected = -om ** 2 * m.ravel() ** 2 * ((1 - 1j * al) - (b1 - 1j * b2))
    assert np.abs(Dm - np.diag(expected)).max() < 1e-9 * np.abs(expected).max()
    D = sp.diags(op.boundary_weights(n))
    DH = (D @ H).toarray()
    assert np.abs(DH - DH.T).max() < 1e-12 * np.abs(DH).max()
    # damping and the outgoing boundary both give Im(D H) >= 0 on the diagonal
    assert np.all(np.diag(DH).imag > 0)


def test_paper_shift_is_M_with_negated_beta1():
    """P = -Lap + beta k^2 (Eq. 6) equals M(beta1 = -b1, beta2 = b2)."""
    n, h, om, al = (6, 5), 10.0, 2 * np.pi * 9, 0.02
    m = np.full(n[::-1], 1 / 2100.0)
    L = op.laplacian_bc(n, h, op.kappa(om, m, al))
    for b1, b2 in [(1.0, 1.0), (0.5, 0.3)]:
        P = L + sp.diags((b1 + 1j * b2) * om ** 2 * m.ravel() ** 2)
        M = op.assemble_M(n, h, m, om, al, -b1, b2)
        assert abs(P - M).max() < 1e-12 * abs(P).max()


# ---------------------------------------------------------------- spectrum (K6, Fig. 2)

def _paper_params():
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as fh:
        return json.load(fh)


def test_dirichlet_spectrum_on_circle():
    """Constant k, Dirichlet, no damping, beta1 = 1: the eigenvalues of M^-1 H
    are s/(s + j beta2 k^2) for real s, so |lambda - 1/2| = 1/2 exactly."""
    n, h, k2 = 30, 1.0 / 31, 300.0
    T = (np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)) / h ** 2
    I = np.eye(n)
    Lap = np.kron(T, I) + np.kron(I, T)
    for b2 in (0.5, 1.0):
        H = Lap - k2 * np.eye(n * n)
        M = Lap - (1.0 - 1j * b2) * k2 * np.eye(n * n)
        lam = np.linalg.eigvals(np.linalg.solve(M, H))
        assert np.abs(np.abs(lam - 0.5) - 0.5).max() < 1e-10


def test_absorbing_spectrum_in_disc_paper_fig2():
    """The paper's 1D spectral experiment (30 Hz, layered well, Fig. 2).

    With the (beta1 - j beta2) reading, the eigenvalues of M^-1 H for the
    paper's beta = (1, 1) and for (1, 0.5) lie in the disc |lambda - 1/2| <=
    1/2 and have positive real parts: they move off the origin and the
    negative real axis, as the paper states. The literal sign of Eq. 6
    (P = -Lap + beta k^2) puts eigenvalues at negative real parts, which
    contradicts that statement; this is why the build takes the other
    reading.
    """
    p = _paper_params()
    om = 2 * np.pi * p["spectrum_frequency_hz"]["value"]
    b1, b2 = p["shift_beta"]["value"]
    n, h, al = 201, 5.0, 0.01
    i = np.arange(n)
    m = 1.0 / np.where(i < n // 3, 1500.0, np.where(i < 2 * n // 3, 2500.0, 3500.0))
    H = op.assemble_H((n,), h, m, om, al).toarray()
    for beta in ((b1, b2), (1.0, 0.5)):
        M = op.assemble_M((n,), h, m, om, al, *beta).toarray()
        lam = np.linalg.eigvals(np.linalg.solve(M, H))
        assert np.abs(lam - 0.5).max() <= 0.5 + 1e-9
        assert lam.real.min() > 0.0
    lam_H = np.linalg.eigvals(H)
    assert lam_H.real.min() < 0.0          # H itself is indefinite
    P_literal = op.assemble_M((n,), h, m, om, al, -b1, b2).toarray()
    lam = np.linalg.eigvals(np.linalg.solve(P_literal, H))
    assert lam.real.min() < -0.1


# ---------------------------------------------------------------- GMRES (Eq. 7)

def test_givens_zeroes_second_component():
    rng = np.random.default_rng(0)
    for _ in range(20):
        a, b = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        c, s, r = gmres.givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        out = G @ np.array([a, b])
        assert abs(out[1]) < 1e-14 * abs(r) and abs(out[0] - r) < 1e-14 * abs(r)
        assert abs(np.linalg.det(G) - 1) < 1e-14 and np.allclose(G.conj().T @ G, np.eye(2))
    c, s, r = gmres.givens(0.0, 2.0 + 1j)
    assert c == 0.0 and abs(r - (2 + 1j)) < 1e-15


def _small_system(n=(9, 7), seed=5, f_hz=12.0):
    rng = np.random.default_rng(seed)
    h, al = 10.0, 0.01
    om = 2 * np.pi * f_hz
    m = 1.0 / rng.uniform(1500, 4500, size=n[::-1])
    H = op.assemble_H(n, h, m, om, al)
    M = op.assemble_M(n, h, m, om, al, 1.0, 0.5)
    N = int(np.prod(n))
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return H, M, f


def test_arnoldi_relation():
    H, M, f = _small_system()
    luM = spla.splu(M.tocsc())
    V, Z, Hb = gmres.arnoldi(lambda x: H @ x, luM.solve, f, 8)
    assert np.abs(H @ Z - V @ Hb).max() < 1e-12 * np.abs(Hb).max()
    # modified Gram-Schmidt keeps the leading vectors orthonormal to rounding;
    # later ones lose orthogonality in proportion to the condition number
    G = V[:, :3].conj().T @ V[:, :3]
    assert np.abs(G - np.eye(3)).max() < 1e-10
    assert np.abs(np.linalg.norm(V, axis=0) - 1.0).max() < 1e-13


def test_gmres_matches_lu_and_residual_decreases():
    H, M, f = _small_system()
    luM = spla.splu(M.tocsc())
    u_lu = spla.splu(H.tocsc()).solve(f)
    r = gmres.gmres_right(lambda x: H @ x, f, 1e-12, 10, 500, Pinv=luM.solve)
    assert r["converged"]
    assert np.linalg.norm(r["x"] - u_lu) < 1e-9 * np.linalg.norm(u_lu)
    assert direct.true_relative_residual(H, f, r["x"]) <= 1e-12
    hist = np.array(r["history"])
    # within each cycle of 10 the least-squares residual never grows
    for c0 in range(0, len(hist), 10):
        seg = hist[c0:c0 + 10]
        assert np.all(np.diff(seg) <= 1e-14)


def test_full_gmres_terminates_in_N_steps():
    H, M, f = _small_system(n=(6, 5))
    N = f.shape[0]
    r = gmres.gmres_right(lambda x: H @ x, f, 1e-10, N, N)
    assert r["converged"] and r["iterations"] <= N


def test_gmres_from_an_initial_guess():
    """Eq. 7 with x0 given: the stopping test stays relative to ||f||, so the
    exact solution as x0 takes no iteration, any x0 reaches the LU solution,
    a close x0 takes fewer iterations than x0 = 0, and f = 0 gives 0."""
    H, M, f = _small_system()
    luM = spla.splu(M.tocsc())
    u_lu = spla.splu(H.tocsc()).solve(f)
    A = lambda x: H @ x  # noqa: E731
    r = gmres.gmres_right(A, f, 1e-10, 10, 500, Pinv=luM.solve, x0=u_lu)
    assert r["converged"] and r["iterations"] == 0 and np.array_equal(r["x"], u_lu)
    rng = np.random.default_rng(3)
    x0 = (rng.standard_normal(f.shape) + 1j * rng.standard_normal(f.shape)) * np.abs(u_lu).max()
    r = gmres.gmres_right(A, f, 1e-10, 10, 500, Pinv=luM.solve, x0=x0)
    assert r["converged"] and np.linalg.norm(r["x"] - u_lu) < 1e-8 * np.linalg.norm(u_lu)
    cold = gmres.gmres_right(A, f, 1e-10, 10, 500, Pinv=luM.solve)
    loose = gmres.gmres_right(A, f, 1e-4, 10, 500, Pinv=luM.solve)
    warm = gmres.gmres_right(A, f, 1e-10, 10, 500, Pinv=luM.solve, x0=loose["x"])
    assert warm["converged"] and 0 < warm["iterations"] < cold["iterations"]
    z = gmres.gmres_right(A, np.zeros_like(f), 1e-10, 10, 500, Pinv=luM.solve, x0=x0)
    assert z["converged"] and z["iterations"] == 0 and not z["x"].any()


def test_preconditioning_cuts_iterations_1d_well():
    """Example section: plain GMRES converges slowly, shifted-Laplace GMRES fast."""
    n, h, om, al = 401, 5.0, 2 * np.pi * 10.0, 0.01
    i = np.arange(n)
    m = 1.0 / np.where(i < n // 3, 1500.0, np.where(i < 2 * n // 3, 2500.0, 3500.0))
    H = op.assemble_H((n,), h, m, om, al)
    M = op.assemble_M((n,), h, m, om, al, 1.0, 0.5)
    f = np.zeros(n, complex)
    f[n // 2] = 1 / h
    luM = spla.splu(M.tocsc())
    rp = gmres.gmres_right(lambda x: H @ x, f, 1e-8, 50, 2000, Pinv=luM.solve)
    r0 = gmres.gmres_right(lambda x: H @ x, f, 1e-8, 50, 400)
    assert rp["converged"] and rp["iterations"] < 100
    assert not r0["converged"]


# ---------------------------------------------------------------- split preconditioning (Eq. 5)

def _krylov_minimiser(B, b, x0_map, k):
    """Brute force: the u = x0_map(K c) over the Krylov basis K = [b, B b, ...,
    B^(k-1) b] that minimises ||b - B K c||_2 (numpy least squares)."""
    K = np.empty((b.shape[0], k), dtype=np.complex128)
    K[:, 0] = b
    for i in range(1, k):
        K[:, i] = B @ K[:, i - 1]
    c = np.linalg.lstsq(B @ K, b, rcond=None)[0]
    return x0_map(K @ c)


@pytest.mark.parametrize("side", ["left", "right", "split"])
def test_split_gmres_minimises_the_preconditioned_residual(side):
    """After k steps (no restart, x0 = 0), GMRES on Ml^-1 A Mr^-1 z = Ml^-1 f
    returns u = Mr^-1 z_k, where z_k minimises the preconditioned residual over
    K_k(Ml^-1 A Mr^-1, Ml^-1 f). This is checked against an explicit Krylov
    basis and numpy least squares, for left, right and two-sided
    preconditioning."""
    H, M, f = _small_system(n=(6, 5))
    Hd, Md = H.toarray(), M.toarray()
    D = np.diag(np.diag(Md))                       # a second, different preconditioner
    Ml, Mr = {"left": (Md, None), "right": (None, Md), "split": (D, Md)}[side]
    Li = np.eye(Hd.shape[0]) if Ml is None else np.linalg.inv(Ml)
    Ri = np.eye(Hd.shape[0]) if Mr is None else np.linalg.inv(Mr)
    B = Li @ Hd @ Ri
    b = Li @ f
    for k in (1, 2, 4, 6):
        r = gmres.gmres_split(lambda x: Hd @ x, f, 1e-300, 100, k,
                              Ml_inv=None if Ml is None else (lambda v: Li @ v),
                              Mr_inv=None if Mr is None else (lambda v: Ri @ v))
        assert r["iterations"] == k
        ref = _krylov_minimiser(B, b, lambda z: Ri @ z, k)
        assert np.linalg.norm(r["x"] - ref) <= 1e-8 * np.linalg.norm(ref), k


def test_left_preconditioning_by_H_itself_takes_one_step():
    H, M, f = _small_system(n=(6, 5))
    lu = spla.splu(H.tocsc())
    r = gmres.gmres_split(lambda x: H @ x, f, 1e-12, 10, 50, Ml_inv=lu.solve)
    assert r["converged"] and r["iterations"] == 1
    assert np.linalg.norm(r["x"] - lu.solve(f)) <= 1e-12 * np.linalg.norm(r["x"])


def test_left_preconditioned_shifted_laplacian_1d_well():
    """The left variant (Ml = P, Mr = I in Eq. 5) on the 1D three-layer well:
    it converges to the LU solution; its preconditioned operator P^-1 H has the
    spectrum of H P^-1, so it needs about as many steps as the right variant."""
    n, h, om, al = 401, 5.0, 2 * np.pi * 10.0, 0.01
    i = np.arange(n)
    m = 1.0 / np.where(i < n // 3, 1500.0, np.where(i < 2 * n // 3, 2500.0, 3500.0))
    H = op.assemble_H((n,), h, m, om, al)
    M = op.assemble_M((n,), h, m, om, al, 1.0, 0.5)
    f = np.zeros(n, complex)
    f[n // 2] = 1 / h
    luM = spla.splu(M.tocsc())
    u_lu = spla.splu(H.tocsc()).solve(f)
    left = gmres.gmres_split(lambda x: H @ x, f, 1e-10, 50, 2000, Ml_inv=luM.solve)
    right = gmres.gmres_right(lambda x: H @ x, f, 1e-10, 50, 2000, Pinv=luM.solve)
    assert left["converged"] and right["converged"]
    assert np.linalg.norm(left["x"] - u_lu) <= 1e-7 * np.linalg.norm(u_lu)
    assert left["true_residuals"][-1] <= 1e-8
    assert 0.5 * right["iterations"] <= left["iterations"] <= 2 * right["iterations"]


# ---------------------------------------------------------------- multigrid pieces

def test_level_sizes_of_reference_grids():
    def dims(n):
        out = [tuple(n)]
        while int(np.prod(n)) > 1500 and mg.can_coarsen(n):
            n = tuple((k + 1) // 2 for k in n)
            out.append(n)
        return out
    assert dims((401, 201))[-1] == (51, 26)
    assert dims((801, 401))[-1] == (51, 26)
    assert dims((257, 129))[-1] == (33, 17)
    assert dims((257, 257, 193))[-1] == (9, 9, 7)
    m = np.full((26, 51), 1 / 2000.0)
    lv = mg.build_levels((51, 26), 80.0, m, 60.0, 0.01, 1.0, 0.5)
    assert len(lv) == 1


@pytest.mark.parametrize("nc", [(5,), (4, 3), (3, 4, 2)])
def test_prolongation_exact_on_multilinear(nc):
    nf = tuple(2 * k - 1 for k in nc)
    rng = np.random.default_rng(0)
    coef = rng.standard_normal(2 ** len(nc)) + 1j * rng.standard_normal(2 ** len(nc))

    def multilinear(n, step):
        X = np.meshgrid(*[np.arange(k) * step for k in n[::-1]], indexing="ij")[::-1]
        out = np.zeros(X[0].shape, complex)
        for mask in range(2 ** len(n)):
            term = np.ones(X[0].shape)
            for a in range(len(n)):
                if mask >> a & 1:
                    term = term * X[a]
            out += coef[mask] * term
        return out.ravel()
    assert np.allclose(mg.prolong(nc, multilinear(nc, 2.0)), multilinear(nf, 1.0), atol=1e-12)


def _as_matrix(fn, n_in):
    N = int(np.prod(n_in))
    cols = [fn(np.eye(N)[:, k]) for k in range(N)]
    return np.array(cols).T


@pytest.mark.parametrize("nc", [(4,), (3, 4), (3, 3, 2)])
def test_restriction_is_scaled_adjoint_of_prolongation(nc):
    """R = Dc^-1 P^T D / 2^d, with D the boundary-halving weights."""
    nf = tuple(2 * k - 1 for k in nc)
    P = _as_matrix(lambda e: mg.prolong(nc, e), nc)
    R = _as_matrix(lambda r: mg.restrict(nf, r), nf)
    D = np.diag(op.boundary_weights(nf))
    Dc = np.diag(op.boundary_weights(nc))
    assert np.abs(R - np.linalg.inv(Dc) @ P.T @ D / 2 ** len(nc)).max() < 1e-14
    assert np.allclose(R @ np.ones(R.shape[1]), 1.0)


def test_jacobi_fixed_point_and_first_sweep():
    rng = np.random.default_rng(2)
    n = (9, 5)
    m = 1 / rng.uniform(1500, 4500, size=n[::-1])
    lv = mg.build_levels(n, 10.0, m, 60.0, 0.01, 1.0, 0.5)
    L = lv[0]
    b = rng.standard_normal(L.M.shape[0]) + 0j
    u = spla.spsolve(L.M.tocsc(), b)
    assert np.allclose(mg.jacobi(L, u, b, 0.8), u, rtol=0, atol=1e-12 * np.abs(u).max())
    assert np.allclose(mg.jacobi(L, 0 * b, b, 0.8), 0.8 * b / L.M.diagonal())


def test_single_level_vcycle_is_exact_solve():
    rng = np.random.default_rng(4)
    n = (10, 6)
    m = 1 / rng.uniform(1500, 4500, size=n[::-1])
    lv = mg.build_levels(n, 10.0, m, 60.0, 0.01, 1.0, 0.5)
    assert len(lv) == 1
    b = rng.standard_normal(60) + 1j * rng.standard_normal(60)
    assert np.allclose(lv[0].M @ mg.vcycle(lv, b), b, atol=1e-12 * np.abs(b).max())


@pytest.mark.parametrize("freq", [0.5, 10.0])
def test_vcycle_contraction(freq):
    """V(1,1) error contraction on the shifted Laplacian, by power iteration.

    Textbook damped-Jacobi / full-weighting / bilinear multigrid contracts by
    about 0.35 per cycle near the Laplace limit; it must stay well below 1
    at 10 Hz.
    """
    n, h = (129, 65), 10.0
    m = np.full(n[::-1], 1 / 2000.0)
    lv = mg.build_levels(n, h, m, 2 * np.pi * freq, 0.01, 1.0, 0.5)
    M = lv[0].M
    e = np.random.default_rng(0).standard_normal(M.shape[0]) + 0j
    for _ in range(25):
        e2 = e - mg.vcycle(lv, M @ e, 1, 1, 0.8)
        rho = np.linalg.norm(e2) / np.linalg.norm(e)
        e = e2 / np.linalg.norm(e2)
    assert rho < 0.45


@pytest.mark.parametrize("freq", [0.5, 10.0])
def test_vcycle_contraction_3d(freq):
    """The same in 3D (33 x 33 x 25 -> 17 x 17 x 13 -> 9 x 9 x 7, trilinear
    interpolation, 27-point full weighting). Damped Jacobi with weight 0.8 on
    the 7-point operator smooths less than in 2D, and the V(1,1) cycle
    contracts by about 0.52. A lopsided weight along one axis of the
    restriction raises that above 0.8."""
    n, h = (33, 33, 25), 10.0
    m = np.full(n[::-1], 1 / 2000.0)
    lv = mg.build_levels(n, h, m, 2 * np.pi * freq, 0.01, 1.0, 0.5)
    assert len(lv) == 3
    M = lv[0].M
    e = np.random.default_rng(0).standard_normal(M.shape[0]) + 0j
    for _ in range(25):
        e2 = e - mg.vcycle(lv, M @ e, 1, 1, 0.8)
        rho = np.linalg.norm(e2) / np.linalg.norm(e)
        e = e2 / np.linalg.norm(e2)
    assert rho < 0.6


def test_vcycle_fgmres_matches_lu_small_2d():
    from workloads import workload
    w = workload("2d_smooth_small")
    m = w.slowness()
    om = w.omega()
    H = op.assemble_H(w.n, w.h, m, om, w.alpha)
    f = w.rhs().ravel()
    u_lu = spla.splu(H.tocsc()).solve(f)
    lv = mg.build_levels(w.n, w.h, m, om, w.alpha, *w.beta)
    r = gmres.gmres_right(lambda x: H @ x, f, 1e-8, 30, 500,
                          Pinv=lambda v: mg.vcycle(lv, v, 1, 1, 0.8))
    assert r["converged"] and r["true_residuals"][-1] <= 1e-8
    assert np.linalg.norm(r["x"] - u_lu) <= 1e-6 * np.linalg.norm(u_lu)


# ---------------------------------------------------------------- block FGMRES

def _block_problem(n=(13, 9), seed=51, s=4):
    rng = np.random.default_rng(seed)
    h, om, al = 10.0, 2 * np.pi * 8.0, 0.05
    m = 1.0 / rng.uniform(1500.0, 4500.0, size=n[::-1])
    H = op.assemble_H(n, h, m, om, al).tocsr()
    M = op.assemble_M(n, h, m, om, al, 1.0, 0.5).tocsc()
    luM = spla.splu(M)
    F = rng.standard_normal((H.shape[0], s)) + 1j * rng.standard_normal((H.shape[0], s))
    return H, luM, F


def test_block_fgmres_with_one_source_is_gmres():
    """A block of one right-hand side is restarted FGMRES: same step count,
    same iterate."""
    H, luM, F = _block_problem(s=1)
    A = lambda X: H @ X  # noqa: E731
    b = gmres.block_fgmres(A, F, 1e-10, 15, 2000, Pinv=luM.solve)
    r = gmres.gmres_right(lambda x: H @ x, F[:, 0], 1e-10, 15, 2000, Pinv=luM.solve)
    assert b["converged"] and r["converged"]
    assert b["iterations"] == r["iterations"]
    assert np.linalg.norm(b["X"][:, 0] - r["x"]) <= 1e-9 * np.linalg.norm(r["x"])


def test_block_fgmres_matches_lu_and_never_trails_single_sources():
    """The block space contains each source's own Krylov space, so after k
    block steps (no restart) every source's residual estimate is at most
    that of its own GMRES after k steps; the solution matches sparse LU."""
    H, luM, F = _block_problem(s=4)
    A = lambda X: H @ X  # noqa: E731
    b = gmres.block_fgmres(A, F, 1e-10, 200, 2000, Pinv=luM.solve)
    assert b["converged"] and b["restarts"] == 1
    X_lu = spla.splu(H.tocsc()).solve(F)
    assert np.linalg.norm(b["X"] - X_lu) <= 1e-8 * np.linalg.norm(X_lu)
    for k in range(F.shape[1]):
        r = gmres.gmres_right(lambda x: H @ x, F[:, k], 1e-10, 200, 2000, Pinv=luM.solve)
        hs = r["history"]
        for step, est in enumerate(b["history"]):
            if step < len(hs):
                assert est[k] <= hs[step] * (1 + 1e-6) + 1e-14
    assert b["iterations"] < min(gmres.gmres_right(lambda x: H @ x, F[:, k], 1e-10, 200, 2000,
                                                    Pinv=luM.solve)["iterations"]
                                 for k in range(F.shape[1]))


def test_block_fgmres_terminates_within_the_block_dimension():
    """Without restart the block Krylov space fills the whole space after
    ceil(N / s) block steps: the solve ends in at most that many."""
    n = (5, 4)
    H, luM, F = _block_problem(n=n, s=5)
    A = lambda X: H @ X  # noqa: E731
    b = gmres.block_fgmres(A, F, 1e-11, 100, 100, Pinv=None)
    assert b["converged"] and b["iterations"] <= int(np.ceil(20 / 5))


def test_block_fgmres_restarts_and_zero_source():
    H, luM, F = _block_problem(s=3)
    F[:, 1] = 0.0
    A = lambda X: H @ X  # noqa: E731
    b = gmres.block_fgmres(A, F, 1e-9, 3, 2000, Pinv=luM.solve)
    assert b["converged"] and b["restarts"] > 1
    assert not b["X"][:, 1].any() or np.abs(b["X"][:, 1]).max() < 1e-12
    X_lu = spla.splu(H.tocsc()).solve(F)
    for k in (0, 2):
        assert np.linalg.norm(b["X"][:, k] - X_lu[:, k]) <= 1e-6 * np.linalg.norm(X_lu[:, k])


# ---------------------------------------------------------------- GCRO-DR (recycling)

def _deflatable(N=300, seed=0):
    """A normal matrix with five eigenvalues in [0.01, 0.05] and the rest in
    [1, 2]: restarted GMRES stalls on the small ones, deflating them helps."""
    rng = np.random.default_rng(seed)
    d = np.concatenate([np.array([0.01, 0.02, 0.03, 0.04, 0.05]), rng.uniform(1, 2, N - 5)]).astype(complex)
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    return Q @ np.diag(d) @ Q.conj().T, rng.standard_normal(N) + 0j


def test_gcrodr_without_recycling_is_gmres():
    H, luM, F = _block_problem(s=1)
    A = lambda x: H @ x  # noqa: E731
    r = gmres.gmres_right(A, F[:, 0], 1e-10, 15, 2000, Pinv=luM.solve)
    g = gmres.gcrodr(A, F[:, 0], 1e-10, 15, 0, 2000, Pinv=luM.solve)
    assert g["iterations"] == r["iterations"] and g["converged"]
    assert np.linalg.norm(g["x"] - r["x"]) <= 1e-9 * np.linalg.norm(r["x"])


def test_gcrodr_deflates_small_eigenvalues_and_recycles():
    """Harmonic Ritz deflation of the five small eigenvalues: GCRO-DR(10, 5)
    needs less than half the steps of GMRES(10) (selecting the largest
    harmonic Ritz values instead, a plausible slip, deflates nothing and
    gains nothing); the recycled space then helps a shifted system; A U = C
    with orthonormal C; the solutions match a dense solve."""
    Am, f = _deflatable()
    A = lambda v: Am @ v  # noqa: E731
    r0 = gmres.gmres_right(A, f, 1e-8, 10, 3000)
    r1 = gmres.gcrodr(A, f, 1e-8, 10, 5, 3000)
    assert r0["converged"] and r1["converged"]
    assert r1["iterations"] < 0.5 * r0["iterations"], (r1["iterations"], r0["iterations"])
    x = np.linalg.solve(Am, f)
    assert np.linalg.norm(r1["x"] - x) <= 1e-6 * np.linalg.norm(x)
    U, C = r1["U"], r1["C"]
    assert np.abs(C.conj().T @ C - np.eye(C.shape[1])).max() <= 1e-10
    assert np.abs(Am @ U - C).max() <= 1e-10 * np.abs(C).max()
    A2m = Am + 0.002 * np.eye(Am.shape[0])
    A2 = lambda v: A2m @ v  # noqa: E731
    fresh = gmres.gcrodr(A2, f, 1e-8, 10, 5, 3000)
    rec = gmres.gcrodr(A2, f, 1e-8, 10, 5, 3000, recycle=r1["recycle"])
    assert rec["converged"] and rec["iterations"] < fresh["iterations"]
    x2 = np.linalg.solve(A2m, f)
    assert np.linalg.norm(rec["x"] - x2) <= 1e-6 * np.linalg.norm(x2)


def test_gcrodr_preconditioned_helmholtz_matches_lu():
    H, luM, F = _block_problem(n=(21, 13), s=1)
    A = lambda x: H @ x  # noqa: E731
    g = gmres.gcrodr(A, F[:, 0], 1e-10, 6, 3, 2000, Pinv=luM.solve)
    assert g["converged"] and g["restarts"] > 1
    x = spla.splu(H.tocsc()).solve(F[:, 0])
    assert np.linalg.norm(g["x"] - x) <= 1e-8 * np.linalg.norm(x)
