"""The multi-frequency batched workload at full size against the oracle.

801 x 401 nodes, h = 7.5 m, the seeded 12-layer model with a 10 % lateral
perturbation, 64 surface sources x {5, 10, 15, 20} Hz (256 solves), complex64
V-cycle with the double-single Arnoldi basis -- the launch configuration the
benchmark times. Per frequency the oracle factors H once by sparse LU (Eq. 4)
and solves a sample of four sources spread over the surface; each must match
the batched GPU solution to 1e-6 relative with a true residual <= 1e-8.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import direct  # noqa: E402
from workloads import workload  # noqa: E402

DEV = "cuda:0"
SAMPLE = (0, 21, 42, 63)


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1712_08740_gb300 import helm as h
    return h


def test_batched_801x401_four_frequencies_match_lu(helm):
    w = workload("2d_batched")
    m = w.slowness()
    ns = len(w.sources)
    F = np.stack([w.rhs(k).ravel() for k in range(ns)])
    Fd = torch.from_numpy(F).to(DEV)
    Ud = torch.empty_like(Fd)
    md = torch.from_numpy(m.ravel().copy()).to(DEV)
    g = helm.Grid(w.n, w.h, restart=w.restart, precond="mg", precision="mixed_ds")
    for fi in range(len(w.freqs)):
        g.set_model(md, w.omega(fi), w.alpha)
        g.set_shift(*w.beta)
        _, its, rr = g.solve_batch(ns, Fd, w.tol, Ud)
        assert (rr <= w.tol).all(), (w.freqs[fi], rr.max())
        U = Ud.cpu().numpy()
        lu = direct.lu_factor_H(w.n, w.h, m, w.omega(fi), w.alpha)
        for k in SAMPLE:
            u_lu = lu.solve(F[k])
            err = np.linalg.norm(U[k] - u_lu) / np.linalg.norm(u_lu)
            assert err <= 1e-6, (w.freqs[fi], k, err, int(its[k]))
    g.close()
