"""GPU parity: every step of the path, called through the C ABI, against the
CPU oracle on the same seeded inputs.

Tolerances. Stencil and V-cycle steps in complex128 repeat the oracle's
arithmetic up to rounding order: 1e-13 (stencil) and 1e-10 (V-cycle, whose
dense coarse inverse carries cond(M_c) * eps). In complex64 the V-cycle
agrees to ~1e-6 relative. Full solves must match the sparse-LU solution
to 1e-6 relative L2 with a true relative residual <= 1e-8 (complex128 outer
loop in both precision forms).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import direct, gmres  # noqa: E402
from oracle import multigrid as mg  # noqa: E402
from oracle import operator as op  # noqa: E402
from workloads import workload  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1712_08740_gb300 import helm as h
    return h


def rand_model(n, seed, lo=1500.0, hi=4500.0):
    rng = np.random.default_rng(seed)
    return 1.0 / rng.uniform(lo, hi, size=tuple(n)[::-1])


def rand_c(N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(N) + 1j * rng.standard_normal(N)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).to(DEV)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


SHAPES = [(37,), (2,), (37, 21), (130, 67), (2, 3), (9, 7, 5), (131, 3, 4)]


@pytest.mark.parametrize("n", SHAPES)
def test_apply_H_matches_oracle(helm, n):
    h, om, al = 10.0, 2 * np.pi * 10.0, 0.01
    m = rand_model(n, 1)
    g = helm.Grid(n, h)
    g.set_model(dev(m), om, al)
    x = rand_c(int(np.prod(n)), 2)
    y = torch.empty(len(x), dtype=torch.complex128, device=DEV)
    g.apply_H(dev(x), y)
    ref = op.assemble_H(n, h, m, om, al) @ x
    assert rel(y.cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("n", SHAPES + [(401, 201)])
def test_apply_H_double_single_matches_oracle(helm, n):
    """H z of the double-single Arnoldi step on complex64 input: the oracle's
    complex128 product of the same complex64 values, to the ~48 bits of the
    double-single result (element by element, relative to the largest)."""
    h, om, al = 10.0, 2 * np.pi * 10.0, 0.01
    m = rand_model(n, 5)
    g = helm.Grid(n, h)
    g.set_model(dev(m), om, al)
    x = rand_c(int(np.prod(n)), 6).astype(np.complex64).astype(np.complex128)
    y = torch.empty(len(x), dtype=torch.complex128, device=DEV)
    g.apply_H_ds(dev(x), y)
    ref = op.assemble_H(n, h, m, om, al) @ x
    y = y.cpu().numpy()
    assert np.abs(y - ref).max() <= 2e-13 * np.abs(ref).max()
    assert rel(y, ref) < 1e-13


def test_unit_vectors_give_dense_H_columns(helm):
    n, h, om, al = (8, 8), 12.0, 2 * np.pi * 9.0, 0.02
    m = rand_model(n, 3)
    g = helm.Grid(n, h)
    g.set_model(m.ravel().copy(), om, al)          # host pointer path
    Hd = op.assemble_H(n, h, m, om, al).toarray()
    N = 64
    y = np.zeros(N, complex)
    for k in range(N):
        e = np.zeros(N, complex)
        e[k] = 1.0
        g.apply_H(e, y)                              # host arrays in and out
        assert np.abs(y - Hd[:, k]).max() <= 1e-15 * np.abs(Hd).max()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-13), ("mixed", 3e-6)])
def test_apply_M_every_level(helm, precision, tol):
    n, h, om, al, b = (129, 65), 10.0, 2 * np.pi * 10.0, 0.01, (1.0, 0.5)
    m = rand_model(n, 4)
    g = helm.Grid(n, h, precision=precision)
    g.set_model(dev(m), om, al)
    g.set_shift(*b)
    levels = mg.build_levels(n, h, m, om, al, *b, coarse_max=1500)
    assert g.num_levels == len(levels)
    for l, L in enumerate(levels):
        nl, hl = g.level_info(l)
        assert nl[:2] == L.n and abs(hl - L.h) < 1e-12
        x = rand_c(L.M.shape[0], 10 + l)
        y = torch.empty(len(x), dtype=torch.complex128, device=DEV)
        g.apply_M(l, dev(x), y)
        assert rel(y.cpu().numpy(), L.M @ x) < tol


@pytest.mark.parametrize("n,nu", [((129, 65), (1, 1)), ((65, 33), (2, 1)), ((33, 17, 9), (1, 2)),
                                  ((101, 51), (0, 1))])
def test_vcycle_matches_oracle_f64(helm, n, nu):
    h, om, al, b, wj = 10.0, 2 * np.pi * 10.0, 0.01, (1.0, 0.5), 0.8
    m = rand_model(n, 5)
    g = helm.Grid(n, h, nu1=nu[0], nu2=nu[1], omega_jacobi=wj)
    g.set_model(dev(m), om, al)
    g.set_shift(*b)
    levels = mg.build_levels(n, h, m, om, al, *b, coarse_max=1500)
    r = rand_c(int(np.prod(n)), 6)
    z = torch.empty(len(r), dtype=torch.complex128, device=DEV)
    g.apply_precond(dev(r), z)
    ref = mg.vcycle(levels, r, nu[0], nu[1], wj)
    assert rel(z.cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("mixed", 2e-4)])
def test_fused_3d_vcycle_every_shape_matches_oracle(helm, precision, tol):
    """The fused 3D V(1,1) level kernels (down: Jacobi from zero + residual +
    full weighting; up: prolongation + Jacobi), every compiled tile shape,
    including the down kernel that marches along z, element-wise against the
    oracle's V-cycle. 65 x 65 x 49 nodes: the first coarse level has 25
    planes, so the z-march (16 coarse planes per block) crosses a block
    boundary, and every level has interior tiles."""
    n, h, om, al, b, wj = (65, 65, 49), 10.0, 2 * np.pi * 10.0, 0.01, (1.0, 0.5), 0.8
    m = rand_model(n, 31)
    g = helm.Grid(n, h, precision=precision, nu1=1, nu2=1, omega_jacobi=wj)
    g.set_model(dev(m), om, al)
    g.set_shift(*b)
    levels = mg.build_levels(n, h, m, om, al, *b, coarse_max=1500)
    assert g.num_levels == len(levels) == 4
    assert levels[1].n[2] > 16
    r = rand_c(int(np.prod(n)), 32)
    ref = mg.vcycle(levels, r, 1, 1, wj)
    rd = dev(r)
    for s in range(helm.helm_num_tile_shapes(3)):
        for lev in range(g.num_levels - 1):
            g.set_tiles(lev, s, s)
        z = torch.empty_like(rd)
        g.apply_precond(rd, z)
        zc = z.cpu().numpy()
        err = rel(zc, ref)
        assert err < tol, (s, err)
        # element by element, relative to the largest entry
        assert np.abs(zc - ref).max() <= 10 * tol * np.abs(ref).max(), s
    g.close()


def test_vcycle_mixed_close_to_oracle(helm):
    n, h, om, al, b = (129, 65), 10.0, 2 * np.pi * 10.0, 0.01, (1.0, 0.5)
    m = rand_model(n, 7)
    g = helm.Grid(n, h, precision="mixed")
    g.set_model(dev(m), om, al)
    g.set_shift(*b)
    levels = mg.build_levels(n, h, m, om, al, *b)
    r = rand_c(int(np.prod(n)), 8)
    z = torch.empty(len(r), dtype=torch.complex128, device=DEV)
    g.apply_precond(dev(r), z)
    assert rel(z.cpu().numpy(), mg.vcycle(levels, r, 1, 1, 0.8)) < 2e-4


def test_single_level_complex64_coarse_solve(helm):
    """A grid no larger than coarse_max has one level: the complex64
    preconditioner is the coarse solve alone (FP32 Gauss-Jordan inverse,
    tensor-core product on a TF32 hi/lo split). It matches M^-1 r to FP32
    accuracy (cond(M) ~ 160 here: ~1.4e-6 for an FP32 inverse); TF32 without
    the split would be ~1e-3 off."""
    n, h, om, al = (33, 17), 10.0, 2 * np.pi * 10.0, 0.01
    m = rand_model(n, 9)
    g = helm.Grid(n, h, precision="mixed")
    g.set_model(dev(m), om, al)
    g.set_shift(1.0, 0.5)
    assert g.num_levels == 1
    r = rand_c(33 * 17, 10)
    z = torch.empty(len(r), dtype=torch.complex128, device=DEV)
    g.apply_precond(dev(r), z)
    M = op.assemble_M(n, h, m, om, al, 1.0, 0.5)
    assert rel(z.cpu().numpy(), direct.spla.splu(M.tocsc()).solve(r)) < 2e-5


def test_exact_precond_is_M_inverse(helm):
    n, h, om, al = (61,), 5.0, 2 * np.pi * 10.0, 0.01
    m = rand_model(n, 9)
    g = helm.Grid(n, h, precond="exact")
    g.set_model(dev(m), om, al)
    g.set_shift(1.0, 0.5)
    r = rand_c(61, 10)
    z = torch.empty(61, dtype=torch.complex128, device=DEV)
    g.apply_precond(dev(r), z)
    M = op.assemble_M(n, h, m, om, al, 1.0, 0.5)
    assert rel(z.cpu().numpy(), direct.spla.splu(M.tocsc()).solve(r)) < 1e-11


def test_true_residual_matches_oracle(helm):
    n, h, om, al = (70, 33), 10.0, 2 * np.pi * 10.0, 0.01
    m = rand_model(n, 11)
    g = helm.Grid(n, h)
    g.set_model(dev(m), om, al)
    f, u = rand_c(70 * 33, 12), rand_c(70 * 33, 13)
    H = op.assemble_H(n, h, m, om, al)
    assert abs(g.true_residual(dev(f), dev(u)) - direct.true_relative_residual(H, f, u)) < 1e-13


# ------------------------------------------------------------------ full solves

def solve_workload(helm, w, precision, precond=None, tol=None, host=False):
    m = w.slowness()
    f = w.rhs()
    g = helm.Grid(w.n, w.h, restart=w.restart, precond=precond or w.precond, precision=precision)
    g.set_model(dev(m), w.omega(), w.alpha)
    g.set_shift(*w.beta)
    if host:
        fu = np.ascontiguousarray(f.ravel())
        u = np.zeros_like(fu)
        _, its, rr = g.solve(fu, tol or w.tol, u)
        return u, its, rr, m, f
    fd = dev(f)
    ud = torch.empty_like(fd)
    _, its, rr = g.solve(fd, tol or w.tol, ud)
    return ud.cpu().numpy(), its, rr, m, f


def test_solve_1d_well_exact_shift(helm):
    w = workload("1d_well")
    u, its, rr, m, f = solve_workload(helm, w, "f64")
    u_lu = direct.lu_solve(w.n, w.h, m, w.omega(), w.alpha, f).ravel()
    assert rr <= 1e-8 and rel(u, u_lu) <= 1e-6
    # the oracle's GMRES with M applied by sparse LU takes 71 iterations
    H = op.assemble_H(w.n, w.h, m, w.omega(), w.alpha)
    M = op.assemble_M(w.n, w.h, m, w.omega(), w.alpha, *w.beta)
    luM = direct.spla.splu(M.tocsc())
    ref = gmres.gmres_right(lambda x: H @ x, f.ravel(), w.tol, w.restart, 5000, Pinv=luM.solve)
    assert abs(its - ref["iterations"]) <= 2


@pytest.mark.parametrize("precision", ["f64", "mixed", "mixed_ds"])
def test_solve_2d_smooth_401x201(helm, precision):
    w = workload("2d_smooth")
    u, its, rr, m, f = solve_workload(helm, w, precision)
    u_lu = direct.lu_solve(w.n, w.h, m, w.omega(), w.alpha, f).ravel()
    assert rr <= 1e-8, rr
    assert rel(u, u_lu) <= 1e-6
    assert its < 200


def test_paper_literal_shift_variant(helm):
    """The paper writes its preconditioner as -Lap + beta k^2 with beta = (1, 1); in the
    build's convention M = -Lap - (b1 - j b2) w^2 m^2 that is (b1, b2) = (-1, 1). Run as a
    variant, it is still a valid right preconditioner: the solve converges to the LU answer,
    but (its spectrum lying off the disc |lambda - 1/2| <= 1/2) it needs more iterations than
    the build's (1, 0.5)."""
    w = workload("2d_smooth_small")
    m = w.slowness()
    f = w.rhs()
    out = {}
    for shift in ((1.0, 0.5), (-1.0, 1.0)):
        g = helm.Grid(w.n, w.h, restart=30)
        g.set_model(dev(m), w.omega(), w.alpha)
        g.set_shift(*shift)
        fd = dev(f)
        ud = torch.empty_like(fd)
        _, its, rr = g.solve(fd, 1e-8, ud)
        out[shift] = (ud.cpu().numpy(), its, rr)
        g.close()
    u_lu = direct.lu_solve(w.n, w.h, m, w.omega(), w.alpha, f).ravel()
    for shift, (u, its, rr) in out.items():
        assert rr <= 1e-8 and rel(u, u_lu) <= 1e-6, shift
    assert out[(-1.0, 1.0)][1] > out[(1.0, 0.5)][1]


def test_solve_host_pointers_equal_device(helm):
    w = workload("2d_smooth_small")
    u1, its1, rr1, _, _ = solve_workload(helm, w, "f64")
    u2, its2, rr2, _, _ = solve_workload(helm, w, "f64", host=True)
    assert its1 == its2 and np.array_equal(u1, u2)


def test_solve_3d_small_mixed(helm):
    w = workload("3d_smooth_small")
    u, its, rr, m, f = solve_workload(helm, w, "mixed")
    u_lu = direct.lu_solve(w.n, w.h, m, w.omega(), w.alpha, f).ravel()
    assert rr <= 1e-8 and rel(u, u_lu) <= 1e-6


@pytest.mark.parametrize("precision", ["f64", "mixed_ds"])
def test_solve_3d_small_other_precisions(helm, precision):
    """The 3D solve in complex128 and with the double-single basis (the form
    the 3D benchmark runs) against sparse LU."""
    w = workload("3d_smooth_small")
    u, its, rr, m, f = solve_workload(helm, w, precision)
    u_lu = direct.lu_solve(w.n, w.h, m, w.omega(), w.alpha, f).ravel()
    assert rr <= 1e-8 and rel(u, u_lu) <= 1e-6


def test_unpreconditioned_matches_oracle_iterations(helm):
    n, h, om, al = (17, 9), 10.0, 2 * np.pi * 6.0, 0.05
    m = rand_model(n, 14)
    f = rand_c(17 * 9, 15)
    g = helm.Grid(n, h, restart=20, precond="none")
    g.set_model(dev(m), om, al)
    g.set_shift(1.0, 0.5)
    u = torch.empty(len(f), dtype=torch.complex128, device=DEV)
    _, its, rr = g.solve(dev(f), 1e-9, u)
    H = op.assemble_H(n, h, m, om, al)
    ref = gmres.gmres_right(lambda x: H @ x, f, 1e-9, 20, 5000)
    assert rr <= 1e-9 and abs(its - ref["iterations"]) <= 3
    assert rel(u.cpu().numpy(), spsolve(H, f)) < 1e-6


def spsolve(H, f):
    return direct.spla.spsolve(H.tocsc(), f)


def test_batch_equals_single(helm):
    w = workload("2d_smooth_small")
    m = w.slowness()
    srcs = [(10, 2), (50, 2), (90, 2), (30, 40)]
    from workloads import point_sources
    F = np.stack([point_sources(w.n, w.h, [s]).ravel() for s in srcs])
    g = helm.Grid(w.n, w.h, restart=30)
    g.set_model(dev(m), w.omega(), w.alpha)
    g.set_shift(*w.beta)
    Fd = dev(F)
    Ud = torch.empty_like(Fd)
    _, its_b, rr_b = g.solve_batch(len(srcs), Fd, 1e-8, Ud)
    Ub = Ud.cpu().numpy().reshape(len(srcs), -1)
    for k in range(len(srcs)):
        fk = dev(F[k])
        uk = torch.empty_like(fk)
        _, its, rr = g.solve(fk, 1e-8, uk)
        assert its == its_b[k]
        assert np.array_equal(Ub[k], uk.cpu().numpy())     # batching does not change arithmetic
        assert rr_b[k] <= 1e-8


# ------------------------------------------------------------------ failure paths (host side)

def test_errors_are_reported(helm):
    n = (33, 17)
    g = helm.Grid(n, 10.0)
    f = dev(rand_c(33 * 17, 1))
    u = torch.empty_like(f)
    with pytest.raises(helm.HelmError) as e:
        g.solve(f, 1e-8, u)
    assert e.value.status == 7                       # solve before model
    g.set_model(dev(rand_model(n, 2)), 60.0, 0.01)
    bad = f.clone()
    bad[5] = complex(float("nan"), 0.0)
    with pytest.raises(helm.HelmError) as e:
        g.solve(bad, 1e-8, u)
    assert e.value.status == 6                       # non-finite right-hand side
    g.set_options(max_iters=3)
    st, its, rr = g.solve(f, 1e-12, u, check=False)
    assert st == 4 and its == 3 and rr > 1e-12       # iteration cap: last iterate returned
    m_bad = rand_model(n, 3)
    m_bad[2, 2] = -1.0
    with pytest.raises(helm.HelmError) as e:
        g.set_model(dev(m_bad), 60.0, 0.01)
    assert e.value.status == 6
    g2 = helm.Grid((80, 60), 10.0)                   # even axes cannot be coarsened
    g2.set_model(dev(rand_model((80, 60), 4)), 60.0, 0.01)
    with pytest.raises(helm.HelmError) as e:
        g2.set_shift(1.0, 0.5)
    assert e.value.status == 8


@pytest.mark.parametrize("precision", ["f64", "mixed", "mixed_ds"])
def test_graph_replay_equals_direct_launches(helm, precision):
    w = workload("2d_smooth_small")
    m = w.slowness()
    from workloads import point_sources
    F = np.stack([point_sources(w.n, w.h, [s]).ravel() for s in [(10, 2), (70, 30), (99, 50)]])
    out = []
    for graphs in (True, False):
        g = helm.Grid(w.n, w.h, restart=12, precision=precision, graphs=graphs)
        g.set_model(dev(m), w.omega(), w.alpha)
        g.set_shift(*w.beta)
        Fd = dev(F)
        Ud = torch.empty_like(Fd)
        _, its, rr = g.solve_batch(3, Fd, 1e-9, Ud)
        out.append((Ud.cpu().numpy(), its, rr))
        assert np.all(rr <= 1e-9)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("reorth", [0, 2])
def test_gram_schmidt_variants_reach_tolerance(helm, reorth):
    """Classical Gram-Schmidt once (default) and the DGKS-selective variant reach
    the tolerance with the same iterations (+-2) as Gram-Schmidt twice."""
    w = workload("2d_smooth_small")
    ref = None
    for mode in (1, reorth):
        g = helm.Grid(w.n, w.h, restart=20, reorth=mode)
        g.set_model(dev(w.slowness()), w.omega(), w.alpha)
        g.set_shift(*w.beta)
        fd = dev(w.rhs())
        ud = torch.empty_like(fd)
        _, its, rr = g.solve(fd, 1e-10, ud)
        assert rr <= 1e-10
        if ref is None:
            ref = (ud.cpu().numpy(), its)
        else:
            assert abs(its - ref[1]) <= 2 and rel(ud.cpu().numpy(), ref[0]) < 1e-8


@pytest.mark.parametrize("precond", ["mg", "none"])
def test_double_single_basis_matches_complex128_basis(helm, precond):
    """The double-single Arnoldi basis reaches the same tolerance with the same
    iteration count (+-2) and a solution within 1e-9 of the complex128-basis
    solution; both match sparse LU to 1e-6."""
    if precond == "mg":
        w = workload("2d_smooth_small")
        n, h, m, om, al, f, restart, tol = w.n, w.h, w.slowness(), w.omega(), w.alpha, w.rhs(), 30, 1e-10
    else:
        n, h, om, al, restart, tol = (17, 9), 10.0, 2 * np.pi * 6.0, 0.05, 20, 1e-10
        m = rand_model(n, 21)
        f = rand_c(17 * 9, 22)
    out = {}
    for prec in ("mixed", "mixed_ds"):
        g = helm.Grid(n, h, restart=restart, precond=precond, precision=prec)
        g.set_model(dev(m), om, al)
        g.set_shift(1.0, 0.5)
        fd = dev(f)
        ud = torch.empty_like(fd)
        _, its, rr = g.solve(fd, tol, ud)
        assert rr <= tol
        out[prec] = (ud.cpu().numpy(), its)
    assert abs(out["mixed"][1] - out["mixed_ds"][1]) <= 2
    assert rel(out["mixed_ds"][0], out["mixed"][0]) < 1e-9
    u_lu = direct.lu_solve(n, h, m, om, al, np.asarray(f).reshape(tuple(n)[::-1])).ravel()
    assert rel(out["mixed_ds"][0], u_lu) < 1e-6


def test_double_single_batch_equals_single(helm):
    w = workload("2d_smooth_small")
    from workloads import point_sources
    F = np.stack([point_sources(w.n, w.h, [s]).ravel() for s in [(10, 2), (60, 20), (95, 49)]])
    g = helm.Grid(w.n, w.h, restart=30, precision="mixed_ds")
    g.set_model(dev(w.slowness()), w.omega(), w.alpha)
    g.set_shift(*w.beta)
    Fd = dev(F)
    Ud = torch.empty_like(Fd)
    _, its_b, rr_b = g.solve_batch(3, Fd, 1e-8, Ud)
    Ub = Ud.cpu().numpy().reshape(3, -1)
    for k in range(3):
        fk = dev(F[k])
        uk = torch.empty_like(fk)
        _, its, rr = g.solve(fk, 1e-8, uk)
        assert its == its_b[k] and np.array_equal(Ub[k], uk.cpu().numpy())


def test_double_single_basis_with_a_long_restart(helm):
    """FGMRES(64): up to 65 basis vectors per Gram-Schmidt pass (nine groups of
    the streamed multi-dot, 65 coefficients per warp in the multi-axpy); the
    double-single solve agrees with the complex128-basis one."""
    w = workload("2d_smooth")
    f = w.rhs().ravel()
    out = {}
    for prec in ("mixed", "mixed_ds"):
        g = helm.Grid(w.n, w.h, restart=64, precision=prec)
        g.set_model(dev(w.slowness()), w.omega(), w.alpha)
        g.set_shift(*w.beta)
        fd = dev(f)
        ud = torch.empty_like(fd)
        _, its, rr = g.solve(fd, 1e-8, ud)
        assert rr <= 1e-8
        out[prec] = (ud.cpu().numpy(), its)
        g.close()
    assert out["mixed"][1] > 31                      # the cycle did grow past 32 vectors
    assert abs(out["mixed"][1] - out["mixed_ds"][1]) <= 2
    assert rel(out["mixed_ds"][0], out["mixed"][0]) < 1e-9


def test_more_than_64_sources_batch_equals_single(helm):
    """70 sources: the tensor-core coarse product takes them in two blocks of
    64 (the second partly filled); every source still equals its single solve."""
    w = workload("2d_smooth_small")
    from workloads import point_sources
    ns = 70
    xs = [1 + (k * 97) // (ns - 1) for k in range(ns)]
    F = np.stack([point_sources(w.n, w.h, [(x, 2 + (k % 5))]).ravel() for k, x in enumerate(xs)])
    g = helm.Grid(w.n, w.h, restart=30, precision="mixed_ds")
    g.set_model(dev(w.slowness()), w.omega(), w.alpha)
    g.set_shift(*w.beta)
    Fd = dev(F)
    Ud = torch.empty_like(Fd)
    _, its_b, rr_b = g.solve_batch(ns, Fd, 1e-8, Ud)
    assert (rr_b <= 1e-8).all()
    Ub = Ud.cpu().numpy().reshape(ns, -1)
    for k in (0, 63, 64, 69):
        fk = dev(F[k])
        uk = torch.empty_like(fk)
        _, its, rr = g.solve(fk, 1e-8, uk)
        assert its == its_b[k] and np.array_equal(Ub[k], uk.cpu().numpy())


def test_double_single_basis_on_a_large_grid(helm):
    """513 x 321 nodes: the double-single multi-dot keeps more per-warp partials
    per vector than the other reductions (161 chunks x 8 warps); the solve
    agrees with the complex128-basis solve and meets the residual bound."""
    from workloads import point_sources, smooth_random
    n, h = (513, 321), 10.0
    c = smooth_random(n, h, seed=4)
    m = (1.0 / c).ravel()
    f = point_sources(n, h, [(256, 2)]).ravel()
    out = {}
    for prec in ("mixed", "mixed_ds"):
        g = helm.Grid(n, h, restart=30, precision=prec)
        g.set_model(dev(m), 2 * np.pi * 10.0, 0.01)
        g.set_shift(1.0, 0.5)
        fd = dev(f)
        ud = torch.empty_like(fd)
        _, its, rr = g.solve(fd, 1e-8, ud)
        assert rr <= 1e-8
        out[prec] = (ud.cpu().numpy(), its)
        g.close()
    assert abs(out["mixed"][1] - out["mixed_ds"][1]) <= 2
    assert rel(out["mixed_ds"][0], out["mixed"][0]) < 1e-9


@pytest.mark.parametrize("precision", ["f64", "mixed", "mixed_ds"])
def test_partial_cycle_update_ignores_unfilled_columns(helm, precision):
    """A cycle that ends before `restart` steps (iteration cap or convergence)
    must not read the unfilled basis columns: they may hold NaN bit patterns
    left in device memory (NaN * 0 = NaN would poison the iterate)."""
    junk = torch.full((256 << 20,), float("nan"), dtype=torch.float32, device=DEV)
    del junk
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    w = workload("2d_smooth_small")
    g = helm.Grid(w.n, w.h, restart=12, precision=precision, max_iters=5)
    g.set_model(dev(w.slowness()), w.omega(), w.alpha)
    g.set_shift(*w.beta)
    fd = dev(w.rhs())
    ud = torch.empty_like(fd)
    st, its, rr = g.solve(fd, 1e-8, ud, check=False)
    assert st == 4 and its == 5 and np.isfinite(rr) and 0 < rr < 1
    assert torch.isfinite(ud).all()
