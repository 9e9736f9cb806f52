"""Tile shapes and the autotuner of the multigrid preconditioner.

Every compiled tile shape of the fused V-cycle kernels must give bitwise the
same preconditioner output (the shape only changes which block computes a
node, not the arithmetic), in every precision form and in 2D and 3D; solves
with tuned shapes must equal solves with the default shapes bitwise; the
autotuner must report only compiled shapes, time every smoother candidate,
and leave a grid whose solves still match the sparse-LU oracle.
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


def grid_for(helm, name, precision):
    w = workload(name)
    g = helm.Grid(w.n, w.h, restart=30, precision=precision)
    g.set_model(dev(w.slowness()), w.omega(), w.alpha)
    g.set_shift(*w.beta)
    return w, g


@pytest.mark.parametrize("name,precision", [("2d_smooth", "f64"), ("2d_smooth", "mixed"),
                                            ("3d_smooth_small", "f64"),
                                            ("3d_smooth_small", "mixed")])
def test_every_tile_shape_gives_the_same_preconditioner(helm, name, precision):
    w, g = grid_for(helm, name, precision)
    assert g.num_levels >= 3
    rng = np.random.default_rng(7)
    r = dev(rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N))
    assert g.get_tiles(0) == (-1, -1)                   # automatic until set
    outs = []
    for s in range(helm.helm_num_tile_shapes(len(w.n))):
        for lev in range(g.num_levels - 1):
            g.set_tiles(lev, s, s)
            assert g.get_tiles(lev) == (s, s)
        z = torch.empty_like(r)
        g.apply_precond(r, z)
        outs.append(z.cpu().numpy())
    assert np.isfinite(outs[0]).all() and np.abs(outs[0]).max() > 0
    for z in outs[1:]:
        assert np.array_equal(z, outs[0])
    g.close()


@pytest.mark.parametrize("precision", ["f64", "mixed_ds"])
def test_solve_with_other_tiles_is_bitwise_identical(helm, precision):
    w, g = grid_for(helm, "2d_smooth", precision)
    f = dev(w.rhs())
    u0 = torch.empty_like(f)
    _, its0, rr0 = g.solve(f, 1e-8, u0)
    ns = helm.helm_num_tile_shapes(2)
    for lev in range(g.num_levels - 1):
        g.set_tiles(lev, (lev + 1) % ns, (lev + 2) % ns)
    u1 = torch.empty_like(f)
    _, its1, rr1 = g.solve(f, 1e-8, u1)
    assert its1 == its0 and rr1 == rr0
    assert torch.equal(u0, u1)
    g.close()


def test_autotune_picks_compiled_shapes_and_keeps_parity(helm):
    w, g = grid_for(helm, "2d_smooth_small", "mixed_ds")
    srcs = [(10, 2), (40, 2), (70, 2), (95, 2)]
    F = np.stack([point_sources(w.n, w.h, [s]).ravel() for s in srcs])
    Fd = dev(F)
    rep = g.autotune(len(srcs), Fd, 1e-8)
    ns = helm.helm_num_tile_shapes(2)
    assert rep["levels"] == g.num_levels - 1 >= 1
    for lev in range(rep["levels"]):
        assert 0 <= rep["down_shape"][lev] < ns and 0 <= rep["up_shape"][lev] < ns
        assert 0 < rep["down_us"][lev] <= rep["down_default_us"][lev]
        assert 0 < rep["up_us"][lev] <= rep["up_default_us"][lev]
        assert g.get_tiles(lev) == (rep["down_shape"][lev], rep["up_shape"][lev])
    assert rep["nu_candidates"] == [(1, 1), (2, 1), (1, 2), (2, 2)]
    assert all(t > 0 for t in rep["nu_ms"]) and all(k > 0 for k in rep["nu_iterations"])
    best = int(np.argmin(rep["nu_ms"]))
    assert (rep["nu1"], rep["nu2"]) == rep["nu_candidates"][best]
    o = helm.helm_get_options(g._g)
    assert (o.nu1, o.nu2) == (rep["nu1"], rep["nu2"])
    # the tuned grid still solves to the oracle's answer
    U = torch.empty_like(Fd)
    _, its, rr = g.solve_batch(len(srcs), Fd, 1e-8, U)
    U = U.cpu().numpy().reshape(len(srcs), -1)
    m = w.slowness()
    for k in range(len(srcs)):
        assert rr[k] <= 1e-8
        u_lu = direct.lu_solve(w.n, w.h, m, w.omega(), w.alpha,
                               F[k].reshape(tuple(w.n)[::-1])).ravel()
        assert rel(U[k], u_lu) < 1e-6
    g.close()


def test_autotune_argument_errors(helm):
    w, g = grid_for(helm, "2d_smooth_small", "f64")
    f = dev(w.rhs())
    with pytest.raises(helm.HelmError) as e:
        helm.helm_autotune(g._g, 1, f, 1e-8, 0)
    assert e.value.status == 1
    with pytest.raises(helm.HelmError) as e:
        helm.helm_autotune(g._g, 1, None, 1e-8, helm.HELM_TUNE_SMOOTHER)
    assert e.value.status == 1
    with pytest.raises(helm.HelmError) as e:
        g.set_tiles(0, helm.helm_num_tile_shapes(2), 0)
    assert e.value.status == 1
    g.set_options(precond="none")
    with pytest.raises(helm.HelmError) as e:
        g.autotune(1, f, 1e-8)
    assert e.value.status == 8
    # tiles only: no right-hand side needed
    g.set_options(precond="mg")
    rep = g.autotune(1, None, 1e-8, tiles=True, smoother=False)
    assert rep["levels"] >= 1 and rep["nu_candidates"] == []
    g.close()


@pytest.mark.parametrize("precision", ["mixed_c64", "mixed", "f64"])
def test_batched_solves_equal_for_every_tile_shape(helm, precision):
    """Shapes whose blocks compute several right-hand sides (2 or 4) change
    which block computes a node and right-hand side, not the arithmetic: a
    batch of 5 sources (so the last block of a 2- or 4-source shape is only
    partly filled) comes out bit for bit the same with every shape."""
    w, g = grid_for(helm, "2d_smooth_small", precision)
    ns = helm.helm_num_tile_shapes(2)
    rbs = [helm.helm_tile_rhs_per_block(2, k, s) for s in range(ns) for k in (0, 1)]
    assert set(rbs) <= {1, 2, 4} and max(rbs) > 1
    srcs = [(5, 2), (30, 9), (55, 2), (80, 30), (97, 2)]
    Fd = dev(np.stack([point_sources(w.n, w.h, [s]).ravel() for s in srcs]))
    U0 = torch.empty_like(Fd)
    _, its0, rr0 = g.solve_batch(len(srcs), Fd, 1e-8, U0)
    assert (rr0 <= 1e-8).all()
    for s in range(ns):
        for lev in range(g.num_levels - 1):
            g.set_tiles(lev, s, (s + 3) % ns)
        U = torch.empty_like(Fd)
        _, its, _ = g.solve_batch(len(srcs), Fd, 1e-8, U)
        assert np.array_equal(its, its0) and torch.equal(U, U0), s
    g.close()
