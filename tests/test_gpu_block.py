"""Block flexible GMRES (helm_options.block = 1) against the oracle.

The tensor-core contractions are checked on their own against numpy in
complex128 (FP32-accurate: TF32 hi/lo split, FP32 accumulation, so the bound
is a few 1e-6 of the scale |V| |W|); the solver against the sparse-LU
solution of every source (1e-6, true residual <= 1e-8) and against the
oracle's block FGMRES for the block-step count.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import direct, gmres  # noqa: E402
from oracle import multigrid as mg  # noqa: E402
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
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def padded(rng, rows, N, ld):
    a = np.zeros((rows, ld), np.complex64)
    a[:, :N] = (rng.standard_normal((rows, N)) + 1j * rng.standard_normal((rows, N))).astype(np.complex64)
    return a


@pytest.mark.parametrize("nv,s,N", [(64, 64, 5151), (200, 64, 80601), (960, 64, 20003), (37, 5, 1003),
                                    (1, 1, 9), (513, 17, 4096)])
def test_block_gram_matches_numpy(helm, nv, s, N):
    rng = np.random.default_rng(nv + s)
    ld = (N + 7) // 8 * 8
    V, W = padded(rng, nv, N, ld), padded(rng, s, N, ld)
    G = helm.helm_block_gram(dev(V), dev(W), N)
    ref = V.astype(np.complex128).conj() @ W.astype(np.complex128).T
    scale = np.sqrt(N) * 2.0            # |V_i| |W_c| for unit-variance entries
    assert np.abs(G - ref).max() <= 5e-6 * scale * np.sqrt(2 * N)


@pytest.mark.parametrize("nv,s,N,alpha", [(64, 64, 5151, 1.0), (320, 64, 80601, 1.0), (64, 64, 20003, 0.0),
                                          (11, 3, 1003, 1.0)])
def test_block_combine_matches_numpy(helm, nv, s, N, alpha):
    rng = np.random.default_rng(nv * 3 + s)
    ld = (N + 7) // 8 * 8
    V, W = padded(rng, nv, N, ld), padded(rng, s, N, ld)
    C = (rng.standard_normal((nv, s)) + 1j * rng.standard_normal((nv, s))) / np.sqrt(nv)
    Wd = dev(W)
    helm.helm_block_combine(dev(V), C, alpha, Wd, N)
    out = Wd.cpu().numpy().astype(np.complex128)
    ref = alpha * W.astype(np.complex128) + (V.astype(np.complex128).T @ C).T
    assert np.abs(out[:, :N] - ref[:, :N]).max() <= 2e-5 * np.abs(ref).max()
    assert not out[:, N:].any()                       # the padding stays zero


def block_grid(helm, w, m, **kw):
    g = helm.Grid(w.n, w.h, restart=kw.pop("restart", 30), precision="mixed", block=True, **kw)
    g.set_model(dev(m.ravel().copy()), w.omega(), w.alpha)
    g.set_shift(*w.beta)
    return g


def test_block_solve_matches_lu(helm):
    w = workload("2d_smooth_small")
    m = w.slowness()
    xs = [2 + (k * 96) // 15 for k in range(16)]
    F = np.stack([point_sources(w.n, w.h, [(x, 2)]).ravel() for x in xs])
    g = block_grid(helm, w, m)
    Fd = dev(F)
    Ud = torch.empty_like(Fd)
    _, its, rr = g.solve_batch(len(xs), Fd, 1e-8, Ud)
    assert (rr <= 1e-8).all(), rr.max()
    lu = direct.lu_factor_H(w.n, w.h, m, w.omega(), w.alpha)
    U = Ud.cpu().numpy()
    for k in range(len(xs)):
        assert rel(U[k], lu.solve(F[k])) <= 1e-6, k
    # one block space for all sources: no more block steps than a source's own FGMRES
    gs = helm.Grid(w.n, w.h, restart=30, precision="mixed")
    gs.set_model(dev(m.ravel().copy()), w.omega(), w.alpha)
    gs.set_shift(*w.beta)
    u1 = torch.empty_like(Fd[0])
    _, its1, _ = gs.solve(Fd[0].contiguous(), 1e-8, u1)
    assert its.max() <= its1, (its, its1)


def test_block_steps_match_the_oracle_block_fgmres(helm):
    """Same block space, same stopping rule: the GPU's block-step count is
    the oracle's (complex128 block FGMRES with the oracle's V-cycle) up to the
    complex64 V-cycle and basis. A complex64 basis holds the Arnoldi relation
    to about 1e-7, so a cycle whose estimate reached 1e-8 leaves a true
    residual near 1e-7 and one short restart finishes the solve: at most half
    again the oracle's steps, never fewer than the oracle's minus two."""
    n, h, om, al, b = (65, 33), 10.0, 2 * np.pi * 8.0, 0.01, (1.0, 0.5)
    rng = np.random.default_rng(61)
    m = 1.0 / rng.uniform(1500.0, 4500.0, size=n[::-1])
    xs = [4 + 8 * k for k in range(8)]
    F = np.stack([point_sources(n, h, [(x, 2)]).ravel() for x in xs])
    g = helm.Grid(n, h, restart=30, precision="mixed", block=True)
    g.set_model(dev(m.ravel().copy()), om, al)
    g.set_shift(*b)
    Fd = dev(F)
    Ud = torch.empty_like(Fd)
    _, its, rr = g.solve_batch(len(xs), Fd, 1e-8, Ud)
    H = op.assemble_H(n, h, m, om, al).tocsr()
    levels = mg.build_levels(n, h, m, om, al, *b, coarse_max=1500)
    ref = gmres.block_fgmres(lambda X: H @ X, F.T, 1e-8, 30, 500,
                             Pinv=lambda r: mg.vcycle(levels, r, 1, 1, 0.8))
    assert ref["converged"] and (rr <= 1e-8).all()
    k = int(its.max())
    assert ref["iterations"] - 2 <= k <= 1.5 * ref["iterations"] + 2, (k, ref["iterations"])
    assert rel(Ud.cpu().numpy(), ref["X"].T) <= 1e-6


def test_block_groups_zero_source_warm_start_and_determinism(helm):
    """70 sources (a full block of 64 and one of 6), a zero source, a warm
    start from the solution (no step), and bitwise repeatability."""
    w = workload("2d_smooth_small")
    m = w.slowness()
    ns = 70
    xs = [1 + (k * 97) // (ns - 1) for k in range(ns)]
    F = np.stack([point_sources(w.n, w.h, [(x, 2 + (k % 5))]).ravel() for k, x in enumerate(xs)])
    F[5] = 0.0
    g = block_grid(helm, w, m)
    Fd = dev(F)
    U1 = torch.empty_like(Fd)
    _, its, rr = g.solve_batch(ns, Fd, 1e-8, U1)
    assert (rr <= 1e-8).all() and its[5] == 0 and not U1[5].any()
    U2 = torch.empty_like(Fd)
    g.solve_batch(ns, Fd, 1e-8, U2)
    assert torch.equal(U1, U2)
    lu = direct.lu_factor_H(w.n, w.h, m, w.omega(), w.alpha)
    U = U1.cpu().numpy()
    for k in (0, 40, 63, 64, 69):
        assert rel(U[k], lu.solve(F[k])) <= 1e-6, k
    U3 = U1.clone()
    _, its3, _ = g.solve_batch(ns, Fd, 1e-8, U3, warm=True)
    assert (its3 == 0).all() and torch.equal(U3, U1)


def test_block_64_sources_401x201_match_lu(helm):
    """The 64-source benchmark batch on the 401 x 201 workload."""
    w = workload("2d_smooth")
    m = w.slowness()
    xs = [int(np.floor((k + 0.5) * (w.n[0] - 1) / 64 + 0.5)) for k in range(64)]
    F = np.stack([point_sources(w.n, w.h, [(x, 2)]).ravel() for x in xs])
    g = block_grid(helm, w, m)
    Fd = dev(F)
    Ud = torch.empty_like(Fd)
    _, its, rr = g.solve_batch(64, Fd, 1e-8, Ud)
    assert (rr <= 1e-8).all()
    lu = direct.lu_factor_H(w.n, w.h, m, w.omega(), w.alpha)
    UL = lu.solve(np.ascontiguousarray(F.T)).T
    U = Ud.cpu().numpy()
    assert max(rel(U[k], UL[k]) for k in range(64)) <= 1e-6


def test_block_options_are_checked(helm):
    w = workload("2d_smooth_small")
    g = helm.Grid(w.n, w.h)
    for kw in ({"precision": "f64"}, {"precision": "mixed_ds"}, {"precision": "mixed", "side": "left"},
               {"precision": "mixed", "restart": 40}, {"precision": "mixed", "precond": "none"}):
        with pytest.raises(helm.HelmError) as e:
            g.set_options(block=True, **kw)
        assert e.value.status == 8
