"""Left and two-sided preconditioning (Eq. 5) on the GPU against the oracle.

Eq. 5 writes the preconditioned system as Ml^-1 H Mr^-1 z = Ml^-1 f with
u = Mr^-1 z; the paper's own choice (Eq. 7) is Ml = I, Mr = M. The library
also runs Ml = M, Mr = I ("left") and Ml = Mr = M ("split"). Both minimise
and stop on the preconditioned residual ||M^-1 (f - H u)|| relative to
||M^-1 f||, as the oracle's gmres_split does. With M applied exactly (its
dense inverse) the GPU's iteration counts must equal the oracle's up to
rounding (+-2), and every solution must match sparse LU.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import direct, gmres  # noqa: E402
from oracle import operator as op  # noqa: E402
from workloads import point_sources, workload  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1712_08740_gb300 import helm as h
    return h


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).to(DEV)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def small_problem():
    n, h, om, al = (61, 41), 10.0, 2 * np.pi * 10.0, 0.01
    rng = np.random.default_rng(41)
    m = 1.0 / rng.uniform(1500.0, 4500.0, size=n[::-1])
    f = point_sources(n, h, [(30, 2)]).ravel()
    return n, h, m, om, al, f


@pytest.mark.parametrize("side", ["left", "split"])
def test_exact_M_matches_oracle_gmres_split(helm, side):
    n, h, m, om, al, f = small_problem()
    tol, restart = 1e-10, 20
    g = helm.Grid(n, h, restart=restart, precond="exact", precision="f64", side=side)
    g.set_model(dev(m), om, al)
    g.set_shift(1.0, 0.5)
    fd = dev(f)
    ud = torch.empty_like(fd)
    _, its, rr = g.solve(fd, tol, ud)
    H = op.assemble_H(n, h, m, om, al)
    luM = direct.lu_factor_M(n, h, m, om, al, 1.0, 0.5)
    ref = gmres.gmres_split(lambda x: H @ x, f, tol, restart, 5000, Ml_inv=luM.solve,
                            Mr_inv=luM.solve if side == "split" else None)
    assert ref["converged"]
    assert abs(its - ref["iterations"]) <= 2, (its, ref["iterations"])
    u = ud.cpu().numpy()
    u_lu = direct.spla.splu(H.tocsc()).solve(f)
    assert rel(u, u_lu) <= 1e-6
    # the reported residual is the true one
    assert abs(rr - direct.true_relative_residual(H, f, u)) <= 1e-12 + 1e-6 * rr


@pytest.mark.parametrize("side", ["left", "split"])
@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_vcycle_sides_match_lu(helm, side, precision):
    w = workload("2d_smooth_small")
    m, f = w.slowness(), w.rhs().ravel()
    g = helm.Grid(w.n, w.h, restart=30, precond="mg", precision=precision, side=side)
    g.set_model(dev(m), w.omega(), w.alpha)
    g.set_shift(*w.beta)
    fd = dev(f)
    ud = torch.empty_like(fd)
    _, its, rr = g.solve(fd, 1e-10, ud)
    u_lu = direct.lu_solve(w.n, w.h, m, w.omega(), w.alpha, f)
    assert rel(ud.cpu().numpy(), u_lu) <= 1e-6
    assert rr <= 1e-6
    # right preconditioning on the same grid: same answer
    g.set_options(side="right")
    ur = torch.empty_like(fd)
    g.solve(fd, 1e-10, ur)
    assert rel(ud.cpu().numpy(), ur.cpu().numpy()) <= 1e-6


def test_left_batch_warm_and_zero_source(helm):
    """Batched left preconditioning: a zero source returns 0, a warm start
    from the solution takes no step, and batch members equal single solves."""
    w = workload("2d_smooth_small")
    m = w.slowness()
    F = np.stack([point_sources(w.n, w.h, [s]).ravel() for s in [(10, 2), (60, 20)]]
                 + [np.zeros(w.unknowns, complex)])
    g = helm.Grid(w.n, w.h, restart=30, precond="mg", precision="f64", side="left")
    g.set_model(dev(m), w.omega(), w.alpha)
    g.set_shift(*w.beta)
    Fd = dev(F)
    Ud = torch.empty_like(Fd)
    _, its, rr = g.solve_batch(3, Fd, 1e-9, Ud)
    U = Ud.cpu().numpy().reshape(3, -1)
    assert its[2] == 0 and not U[2].any()
    for k in range(2):
        uk = torch.empty_like(dev(F[k]))
        _, itk, _ = g.solve(dev(F[k]), 1e-9, uk)
        assert itk == its[k] and np.array_equal(uk.cpu().numpy(), U[k])
    U2 = Ud.clone()
    _, its2, _ = g.solve_batch(3, Fd, 1e-9, U2, warm=True)
    assert (its2 == 0).all() and torch.equal(U2, Ud)


def test_double_single_basis_rejects_left(helm):
    w = workload("2d_smooth_small")
    g = helm.Grid(w.n, w.h)
    with pytest.raises(helm.HelmError) as e:
        g.set_options(precision="mixed_ds", side="left")
    assert e.value.status == 8
