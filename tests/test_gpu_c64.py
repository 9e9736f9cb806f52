"""The complex64-basis form (precision "mixed_c64") against sparse LU and
against the double-single basis.

The basis vectors are stored in complex64; w = H z and its Gram-Schmidt
update stay double-single until v_{j+1} is rounded, and the Hessenberg least
squares, the solution and the true residual stay complex128. A restarted
cycle then only has to reach about 1e-7 of its own starting residual, far
above the rounding of the basis, so the step counts match the double-single
basis to within a step or two and every solution matches LU to 1e-6.
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
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def grid(helm, w, m, precision, **kw):
    g = helm.Grid(w.n, w.h, restart=kw.pop("restart", w.restart), precision=precision, **kw)
    g.set_model(dev(m.ravel().copy()), w.omega(), w.alpha)
    g.set_shift(*w.beta)
    return g


def surface_batch(w, count):
    xs = [int(np.floor((k + 0.5) * (w.n[0] - 1) / count + 0.5)) for k in range(count)]
    return np.stack([point_sources(w.n, w.h, [(x, 2)]).ravel() for x in xs])


def test_single_solve_401x201_matches_lu_and_double_single(helm):
    w = workload("2d_smooth")
    m = w.slowness()
    f = w.rhs().ravel()
    out = {}
    for prec in ("mixed_c64", "mixed_ds"):
        g = grid(helm, w, m, prec)
        u = torch.empty(f.size, dtype=torch.complex128, device=DEV)
        _, its, rr = g.solve(dev(f), 1e-8, u)
        out[prec] = (its, rr, u.cpu().numpy())
        g.close()
    its, rr, u = out["mixed_c64"]
    assert rr <= 1e-8
    assert abs(its - out["mixed_ds"][0]) <= 2, (its, out["mixed_ds"][0])
    assert rel(u, direct.lu_solve(w.n, w.h, m, w.omega(), w.alpha, f)) <= 1e-6


def test_64_sources_401x201_match_lu(helm):
    w = workload("2d_smooth")
    m = w.slowness()
    F = surface_batch(w, 64)
    Fd = dev(F)
    its = {}
    for prec in ("mixed_c64", "mixed_ds"):
        g = grid(helm, w, m, prec)
        Ud = torch.empty_like(Fd)
        _, it, rr = g.solve_batch(64, Fd, 1e-8, Ud)
        assert (rr <= 1e-8).all(), prec
        its[prec] = it.copy()
        if prec == "mixed_c64":
            U = Ud.cpu().numpy()
        g.close()
    assert (its["mixed_c64"] <= its["mixed_ds"] + 2).all(), (its["mixed_c64"], its["mixed_ds"])
    lu = direct.lu_factor_H(w.n, w.h, m, w.omega(), w.alpha)
    UL = lu.solve(np.ascontiguousarray(F.T)).T
    assert max(rel(U[k], UL[k]) for k in range(64)) <= 1e-6


def test_batch_equals_single_and_graphs_do_not_change_bits(helm):
    w = workload("2d_smooth_small")
    m = w.slowness()
    F = np.stack([point_sources(w.n, w.h, [s]).ravel() for s in [(10, 2), (60, 20), (95, 49), (50, 2)]])
    Fd = dev(F)
    g = grid(helm, w, m, "mixed_c64")
    Ud = torch.empty_like(Fd)
    _, its_b, rr_b = g.solve_batch(4, Fd, 1e-9, Ud)
    assert (rr_b <= 1e-9).all()
    for q in range(4):
        uq = torch.empty_like(Fd[q])
        _, its, _ = g.solve(Fd[q].contiguous(), 1e-9, uq)
        assert its == its_b[q] and torch.equal(uq, Ud[q]), q
    g2 = grid(helm, w, m, "mixed_c64", graphs=False)
    U2 = torch.empty_like(Fd)
    g2.solve_batch(4, Fd, 1e-9, U2)
    assert torch.equal(U2, Ud)
    # warm start from the solution: no step, the same bits
    U3 = Ud.clone()
    _, its3, _ = g.solve_batch(4, Fd, 1e-9, U3, warm=True)
    assert (its3 == 0).all() and torch.equal(U3, Ud)
    g.close()
    g2.close()


def test_3d_small_matches_lu(helm):
    w = workload("3d_smooth_small")
    m = w.slowness()
    f = w.rhs().ravel()
    g = grid(helm, w, m, "mixed_c64")
    u = torch.empty(f.size, dtype=torch.complex128, device=DEV)
    _, its, rr = g.solve(dev(f), 1e-8, u)
    assert rr <= 1e-8
    assert rel(u.cpu().numpy(), direct.lu_solve(w.n, w.h, m, w.omega(), w.alpha, f)) <= 1e-6
    g.close()


def test_autotuned_tiles_keep_the_result(helm):
    """Tile shapes do not change the arithmetic: the tuned grid reproduces the
    untuned solve bit for bit."""
    w = workload("2d_smooth")
    m = w.slowness()
    Fd = dev(surface_batch(w, 8))
    g = grid(helm, w, m, "mixed_c64")
    U1 = torch.empty_like(Fd)
    g.solve_batch(8, Fd, 1e-8, U1)
    g.autotune(8, None, 1e-8, tiles=True, smoother=False)
    U2 = torch.empty_like(Fd)
    _, its, rr = g.solve_batch(8, Fd, 1e-8, U2)
    assert (rr <= 1e-8).all() and torch.equal(U1, U2)
    g.close()


def test_options_are_checked(helm):
    w = workload("2d_smooth_small")
    g = helm.Grid(w.n, w.h)
    for kw in ({"side": "left"}, {"side": "split"}, {"reorth": 1}, {"precond": "none"}):
        with pytest.raises(helm.HelmError) as e:
            g.set_options(precision="mixed_c64", **kw)
        assert e.value.status == 8
    g.set_model(dev(w.slowness().ravel().copy()), w.omega(), w.alpha)
    g.set_options(precision="mixed_c64")
    with pytest.raises(helm.HelmError) as e:
        g.set_density(dev(np.ones(w.unknowns)))
    assert e.value.status == 8
    g.close()
