"""The allocation-free residual entry point (helm_true_residual_noalloc).

Callers that cannot call cudaMalloc -- a serving process that reserved the
GPU's memory up front for its own pool, or a caller that must not stall other
streams on cudaMalloc/cudaFree -- use this variant; it keeps its scratch in a
static device array of the library. These tests call it through the C ABI
and compare it with the allocating helm_true_residual on the same device
data, on two calls in a row, in 1D, 2D and 3D. The file is collected last so
that a stop-at-first-failure run has already run every other test; it also
passes alone in a fresh process (the first call there performs the one-time
look-up of the array's address).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1712_08740_gb300 import helm as h
    return h


def _grid(helm, n=(130, 67), h=10.0, seed=0):
    rng = np.random.default_rng(seed)
    m = 1.0 / rng.uniform(1500.0, 4500.0, size=n[::-1])
    g = helm.Grid(n, h)
    g.set_model(torch.from_numpy(m.ravel().copy()).to("cuda:0"), 2 * np.pi * 10.0, 0.01)
    return g


def _pairs(nrhs, N, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((2, nrhs, N)) + 1j * rng.standard_normal((2, nrhs, N))
    return torch.from_numpy(a[0]).to("cuda:0"), torch.from_numpy(a[1]).to("cuda:0")


# 1D, 2D and 3D grids: the kernel carries its own stencil for each dimension
# (boundary faces, corner counts, plane strides)
@pytest.mark.parametrize("n", [(101,), (130, 67), (17, 13, 9)])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_noalloc_residual_matches_allocating_entry_point(helm, n, nrhs):
    g = _grid(helm, n=n)
    for call in range(2):                       # two calls in a row, new data each time
        F, U = _pairs(nrhs, g.N, seed=10 + call)
        rel = helm.helm_true_residual_noalloc(g, nrhs, F, U)
        for k in range(nrhs):
            ref = g.true_residual(F[k].contiguous(), U[k].contiguous())
            assert abs(rel[k] - ref) <= 1e-12 * ref


def test_noalloc_residual_of_a_solution(helm):
    g = _grid(helm, n=(65, 33), seed=3)
    f = torch.zeros(g.N, dtype=torch.complex128, device="cuda:0")
    f[2 * 65 + 32] = 1.0 / 100.0
    u = torch.empty_like(f)
    g.solve(f, 1e-9, u)
    rel = helm.helm_true_residual_noalloc(g, 1, f, u)
    assert rel[0] <= 1e-9 and abs(rel[0] - g.true_residual(f, u)) <= 1e-12


def test_noalloc_rejects_what_it_cannot_serve(helm):
    g = _grid(helm, n=(9, 7))
    F, U = _pairs(65, g.N, seed=1)
    with pytest.raises(helm.HelmError) as e:
        helm.helm_true_residual_noalloc(g, 65, F, U)
    assert e.value.status == 1 and "static scratch" in e.value.message
    fh = np.zeros(g.N, dtype=np.complex128)
    with pytest.raises(helm.HelmError) as e:
        helm.helm_true_residual_noalloc(g, 1, fh, fh)   # host arrays are not staged
    assert e.value.status == 1
    with pytest.raises(ValueError):                      # too short for nrhs right-hand sides
        helm.helm_true_residual_noalloc(g, 2, F[0].contiguous(), U[0].contiguous())
