"""Warm start: restarted FGMRES (Eq. 7) from a given initial guess x0 instead
of 0, through helm_solve_batch_warm. The answer is the same unique u = H^-1 f
(the sparse-LU oracle), the stopping test stays relative to ||f||, and a good
x0 saves iterations: the use in a frequency sweep, where the solution at the
previous frequency starts the next solve.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import direct  # noqa: E402
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


def grid(helm, w, precision, omega=None):
    g = helm.Grid(w.n, w.h, restart=30, precision=precision)
    g.set_model(dev(w.slowness()), w.omega() if omega is None else omega, w.alpha)
    g.set_shift(*w.beta)
    return g


@pytest.mark.parametrize("precision", ["f64", "mixed_ds"])
def test_warm_start_from_the_solution_takes_no_iteration(helm, precision):
    w = workload("2d_smooth_small")
    g = grid(helm, w, precision)
    fd = dev(w.rhs())
    ud = torch.empty_like(fd)
    _, its, rr = g.solve(fd, 1e-8, ud)
    assert its > 0 and rr <= 1e-8
    u_cold = ud.cpu().numpy()
    _, its_w, rr_w = g.solve(fd, 1e-8, ud, warm=True)
    assert its_w == 0 and rr_w <= 1e-8
    assert np.array_equal(ud.cpu().numpy(), u_cold)      # x0 returned as it was
    g.close()


@pytest.mark.parametrize("precision", ["f64", "mixed", "mixed_ds"])
def test_warm_start_from_a_loose_solution(helm, precision):
    w = workload("2d_smooth_small")
    g = grid(helm, w, precision)
    f = w.rhs()
    fd = dev(f)
    ud = torch.empty_like(fd)
    _, its_cold, _ = g.solve(fd, 1e-8, ud)
    _, its_loose, rr_loose = g.solve(fd, 1e-3, ud)
    assert 1e-8 < rr_loose <= 1e-3
    _, its_warm, rr = g.solve(fd, 1e-8, ud, warm=True)
    u_lu = direct.lu_solve(w.n, w.h, w.slowness(), w.omega(), w.alpha, f).ravel()
    assert rr <= 1e-8 and rel(ud.cpu().numpy(), u_lu) <= 1e-6
    assert 0 < its_warm < its_cold, (its_warm, its_cold)
    g.close()


def test_frequency_sweep_warm_start(helm):
    """Sources solved at 10 Hz start the solve at 10.2 Hz; the result is the
    LU solution at 10.2 Hz whatever the start."""
    w = workload("2d_smooth_small")
    m = w.slowness()
    F = np.stack([point_sources(w.n, w.h, [s]).ravel() for s in [(20, 2), (50, 2), (80, 2)]])
    Fd = dev(F)
    Ud = torch.empty_like(Fd)
    om0, om1 = 2 * np.pi * 10.0, 2 * np.pi * 10.2
    g = grid(helm, w, "mixed_ds", om0)
    g.solve_batch(3, Fd, 1e-8, Ud)
    g.set_model(dev(m), om1, w.alpha)
    g.set_shift(*w.beta)
    _, its, rr = g.solve_batch(3, Fd, 1e-8, Ud, warm=True)
    U = Ud.cpu().numpy().reshape(3, -1)
    for k in range(3):
        u_lu = direct.lu_solve(w.n, w.h, m, om1, w.alpha, F[k]).ravel()
        assert rr[k] <= 1e-8 and rel(U[k], u_lu) <= 1e-6, k
    g.close()


def test_warm_batch_host_arrays_zero_source_and_non_finite_guess(helm):
    w = workload("2d_smooth_small")
    m = w.slowness()
    f = w.rhs().ravel()
    F = np.stack([f, np.zeros_like(f), np.roll(f, 7)])
    rng = np.random.default_rng(5)
    X0 = (rng.standard_normal(F.shape) + 1j * rng.standard_normal(F.shape)) * np.abs(f).max()
    U = X0.copy()
    g = grid(helm, w, "f64")
    _, its, rr = g.solve_batch(3, F, 1e-8, U, warm=True)
    assert its[1] == 0 and not U[1].any()                # f = 0: u = 0 whatever x0 was
    for k in (0, 2):
        u_lu = direct.lu_solve(w.n, w.h, m, w.omega(), w.alpha, F[k]).ravel()
        assert rr[k] <= 1e-8 and rel(U[k], u_lu) <= 1e-6, k
    bad = X0.copy()
    bad[2, 11] = complex(np.inf, 0.0)
    with pytest.raises(helm.HelmError) as e:
        g.solve_batch(3, F, 1e-8, bad, warm=True)
    assert e.value.status == 6                           # non-finite initial guess
    g.close()
