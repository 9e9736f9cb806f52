"""The bounded waits of the streamed double-single Arnoldi kernels.

Every wait in those kernels gives up after a time limit instead of spinning
forever; a wait that runs out turns the kernel's results into NaN, which the
solver reports as HELM_ERR_BREAKDOWN. Here the consumers' limit is cut to
1 ns (helm_set_wait_limit_ns), so their first wait for a tile copy that has
not landed yet runs out -- with every copy valid and landing: nothing
faults, and the producers still wait (at the default limit) for the copies
they issued before their blocks exit. The grid must stay usable: with the
default limit restored, the same solve reproduces its earlier result
bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


@pytest.mark.parametrize("precision", ["mixed_ds", "mixed_c64"])
@pytest.mark.parametrize("graphs", [True, False])
def test_wait_timeout_reports_breakdown_and_grid_stays_usable(helm, graphs, precision):
    """The double-single basis and the complex64 basis stream their tiles
    through the same bounded-wait ring."""
    w = workload("2d_smooth_small")
    g = helm.Grid(w.n, w.h, restart=30, precision=precision, graphs=graphs)
    g.set_model(torch.from_numpy(w.slowness().ravel().copy()).to(DEV), w.omega(), w.alpha)
    g.set_shift(*w.beta)
    fd = torch.from_numpy(w.rhs().ravel().copy()).to(DEV)
    u0 = torch.empty_like(fd)
    st0, its0, rr0 = g.solve(fd, 1e-8, u0)
    assert st0 == 0 and rr0 <= 1e-8
    u1 = torch.empty_like(fd)
    helm.helm_set_wait_limit_ns(1)
    try:
        st1, _, _ = g.solve(fd, 1e-8, u1, check=False)
    finally:
        helm.helm_set_wait_limit_ns(0)
    torch.cuda.synchronize()                        # the context is intact
    assert st1 == 5                                 # HELM_ERR_BREAKDOWN
    u2 = torch.empty_like(fd)
    st2, its2, rr2 = g.solve(fd, 1e-8, u2)
    assert st2 == 0 and its2 == its0 and rr2 == rr0
    assert torch.equal(u2, u0)
    g.close()
