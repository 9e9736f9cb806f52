"""Variable density (Eq. 1) on the GPU against the oracle.

-div(rho grad u) - omega^2 m^2 (1 - j alpha) u = f with face-averaged rho and
the absorbing boundary at the local wavenumber kappa / sqrt(rho). Every step
is compared with the oracle's node-by-node operator (oracle/density.py):
H apply in 1D/2D/3D (complex128, 1e-13), M on every multigrid level (1e-13
complex128, 3e-6 complex64), one V-cycle (1e-10 / 2e-4) and full solves
against sparse LU of H_rho (1e-6 with a true residual <= 1e-8), the same
tolerances as the constant-density tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import density  # noqa: E402
from oracle import direct  # noqa: E402
from oracle import multigrid as mg  # noqa: E402
from workloads import point_sources, smooth_random, workload  # noqa: E402

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


def rand_field(n, seed, lo, hi):
    return np.random.default_rng(seed).uniform(lo, hi, size=tuple(n)[::-1])


def seeded_rho(n, h, seed=7):
    """A smooth density-like coefficient in [1.0, 2.5] (Gaussian-smoothed
    noise with a 200 m correlation length, seeded)."""
    return smooth_random(n, h, corr_len=200.0, vmin=1.0, vmax=2.5, seed=seed)


@pytest.mark.parametrize("n", [(37,), (2,), (37, 21), (130, 67), (2, 3), (9, 7, 5), (19, 6, 4)])
def test_apply_H_with_rho_matches_oracle(helm, n):
    h, om, al = 10.0, 2 * np.pi * 10.0, 0.01
    m = 1.0 / rand_field(n, 1, 1500.0, 4500.0)
    rho = rand_field(n, 2, 0.5, 3.0)
    g = helm.Grid(n, h)
    g.set_model(dev(m), om, al)
    g.set_density(dev(rho))
    N = int(np.prod(n))
    rng = np.random.default_rng(3)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    y = torch.empty(N, dtype=torch.complex128, device=DEV)
    g.apply_H(dev(x), y)
    ref = density.assemble_H_rho(n, h, m, rho, om, al) @ x
    assert rel(y.cpu().numpy(), ref) < 1e-13
    g.close()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-13), ("mixed", 3e-6)])
def test_apply_M_with_rho_every_level(helm, precision, tol):
    n, h, om, al, b = (129, 65), 10.0, 2 * np.pi * 10.0, 0.01, (1.0, 0.5)
    m = 1.0 / rand_field(n, 4, 1500.0, 4500.0)
    rho = seeded_rho(n, h)
    g = helm.Grid(n, h, precision=precision)
    g.set_model(dev(m), om, al)
    g.set_density(rho.ravel().copy())                     # host pointer path
    g.set_shift(*b)
    levels = density.build_levels_rho(n, h, m, rho, om, al, *b, coarse_max=1500)
    assert g.num_levels == len(levels) >= 3
    rng = np.random.default_rng(5)
    for l, L in enumerate(levels):
        x = rng.standard_normal(L.M.shape[0]) + 1j * rng.standard_normal(L.M.shape[0])
        y = torch.empty(len(x), dtype=torch.complex128, device=DEV)
        g.apply_M(l, dev(x), y)
        assert rel(y.cpu().numpy(), L.M @ x) < tol, l
    g.close()


@pytest.mark.parametrize("n,precision,tol", [((129, 65), "f64", 1e-10), ((129, 65), "mixed", 2e-4),
                                             ((33, 17, 13), "f64", 1e-10)])
def test_vcycle_with_rho_matches_oracle(helm, n, precision, tol):
    h, om, al, b, wj = 10.0, 2 * np.pi * 10.0, 0.01, (1.0, 0.5), 0.8
    m = 1.0 / rand_field(n, 6, 1500.0, 4500.0)
    rho = seeded_rho(n, h, seed=8)
    g = helm.Grid(n, h, precision=precision, omega_jacobi=wj)
    g.set_model(dev(m), om, al)
    g.set_density(dev(rho))
    g.set_shift(*b)
    levels = density.build_levels_rho(n, h, m, rho, om, al, *b, coarse_max=1500)
    rng = np.random.default_rng(9)
    N = int(np.prod(n))
    r = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    z = torch.empty(N, dtype=torch.complex128, device=DEV)
    g.apply_precond(dev(r), z)
    assert rel(z.cpu().numpy(), mg.vcycle(levels, r, 1, 1, wj)) < tol
    g.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_solve_with_rho_matches_lu(helm, precision):
    w = workload("2d_smooth_small")
    m = w.slowness()
    rho = seeded_rho(w.n, w.h)
    f = w.rhs().ravel()
    g = helm.Grid(w.n, w.h, restart=30, precision=precision)
    g.set_model(dev(m), w.omega(), w.alpha)
    g.set_density(dev(rho))
    g.set_shift(*w.beta)
    fd = dev(f)
    ud = torch.empty_like(fd)
    _, its, rr = g.solve(fd, 1e-8, ud)
    H = density.assemble_H_rho(w.n, w.h, m, rho, w.omega(), w.alpha)
    u_lu = direct.spla.splu(H.tocsc()).solve(f)
    u = ud.cpu().numpy()
    assert rr <= 1e-8 and rel(u, u_lu) <= 1e-6
    assert abs(rr - direct.true_relative_residual(H, f, u)) <= 1e-12
    g.close()


def test_solve_with_rho_401x201_matches_lu(helm):
    """The 401 x 201 workload of the plain benchmark with a seeded rho."""
    w = workload("2d_smooth")
    m = w.slowness()
    rho = seeded_rho(w.n, w.h)
    f = w.rhs().ravel()
    g = helm.Grid(w.n, w.h, restart=30, precision="f64")
    g.set_model(dev(m), w.omega(), w.alpha)
    g.set_density(dev(rho))
    g.set_shift(*w.beta)
    fd = dev(f)
    ud = torch.empty_like(fd)
    _, its, rr = g.solve(fd, 1e-8, ud)
    H = density.assemble_H_rho(w.n, w.h, m, rho, w.omega(), w.alpha)
    u_lu = direct.spla.splu(H.tocsc()).solve(f)
    assert rr <= 1e-8 and rel(ud.cpu().numpy(), u_lu) <= 1e-6
    g.close()


def test_unit_rho_equals_constant_density(helm):
    """rho = 1 everywhere solves Eq. 2 (through the general V-cycle kernels);
    removing the density returns to the fused path; both match."""
    w = workload("2d_smooth_small")
    f = dev(w.rhs())
    g = helm.Grid(w.n, w.h, restart=30)
    g.set_model(dev(w.slowness()), w.omega(), w.alpha)
    g.set_shift(*w.beta)
    u0 = torch.empty_like(f)
    g.solve(f, 1e-10, u0)
    g.set_density(dev(np.ones(w.unknowns)))
    u1 = torch.empty_like(f)
    g.solve(f, 1e-10, u1)
    g.set_density(None)
    u2 = torch.empty_like(f)
    g.solve(f, 1e-10, u2)
    assert rel(u1.cpu().numpy(), u0.cpu().numpy()) < 1e-8
    assert torch.equal(u2, u0)
    g.close()


def test_batch_with_rho_equals_single(helm):
    w = workload("2d_smooth_small")
    F = np.stack([point_sources(w.n, w.h, [s]).ravel() for s in [(10, 2), (60, 20), (95, 49)]])
    g = helm.Grid(w.n, w.h, restart=30, precision="mixed")
    g.set_model(dev(w.slowness()), w.omega(), w.alpha)
    g.set_density(dev(seeded_rho(w.n, w.h)))
    g.set_shift(*w.beta)
    Fd = dev(F)
    Ud = torch.empty_like(Fd)
    _, its_b, rr_b = g.solve_batch(3, Fd, 1e-8, Ud)
    Ub = Ud.cpu().numpy().reshape(3, -1)
    for k in range(3):
        uk = torch.empty_like(dev(F[k]))
        _, its, _ = g.solve(dev(F[k]), 1e-8, uk)
        assert its == its_b[k] and np.array_equal(Ub[k], uk.cpu().numpy())
    g.close()


def test_density_errors(helm):
    n = (33, 17)
    g = helm.Grid(n, 10.0)
    g.set_model(dev(1.0 / rand_field(n, 1, 1500.0, 4500.0)), 60.0, 0.01)
    bad = np.ones(33 * 17)
    bad[40] = 0.0
    with pytest.raises(helm.HelmError) as e:
        g.set_density(dev(bad))
    assert e.value.status == 6
    bad[40] = np.nan
    with pytest.raises(helm.HelmError) as e:
        g.set_density(bad)
    assert e.value.status == 6
    g.set_density(dev(np.ones(33 * 17)))
    with pytest.raises(helm.HelmError) as e:
        g.set_options(precision="mixed_ds")
    assert e.value.status == 8
    x = dev(np.ones(33 * 17, complex))
    with pytest.raises(helm.HelmError) as e:
        g.apply_H_ds(x, torch.empty_like(x))
    assert e.value.status == 8
    g.close()
