"""Grids solving at the same time on their own streams do not change each
other's results.

Each grid owns its buffers and stream, so a batch must come out bit for bit
the same whether it runs alone or while other grids' kernels share the SMs.
Kernels from other streams then run on the same SMs as the solve's own
blocks, and leave their data in shared memory where this solve's next blocks
start: a block that reads a shared-memory word before its own threads have
set it sees that data. The batches here have 40 to 64 sources, so every warp
of the tensor-core coarse product (eight sources per warp) stages a slice,
and several problems run in four threads at once, twice each."""
import math
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads import point_sources, smooth_random  # noqa: E402


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1712_08740_gb300 import helm as h
    return h


def problems():
    out = []
    for t, n in enumerate([(257, 129), (129, 65), (257, 129), (193, 97)]):
        m = (1.0 / smooth_random(n, 10.0, seed=1000 * t + n[0])).ravel()
        count = 64 - 8 * t
        xs = [2 + (k * (n[0] - 5)) // (count - 1) for k in range(count)]
        F = np.stack([point_sources(n, 10.0, [(x, 2)]).ravel() for x in xs])
        out.append((n, m, F))
    return out


def solve(helm, g, p):
    n, m, F = p
    g.set_model(m.copy(), 2 * math.pi * 15.0, 0.01)
    g.set_shift(1.0, 0.5)
    U = np.zeros_like(F)
    st, its, _ = g.solve_batch(F.shape[0], F, 1e-8, U, check=False)
    return st, its.copy(), U


@pytest.mark.parametrize("precision", ["mixed_c64", "mixed_ds", "mixed"])
def test_concurrent_grids_match_serial(helm, precision):
    probs = problems()
    stream = torch.cuda.Stream()
    ref = []
    for p in probs:
        g = helm.Grid(p[0], 10.0, precision=precision)
        g.set_stream(stream.cuda_stream)
        ref.append(solve(helm, g, p))
        g.close()
        assert ref[-1][0] == 0
    out, errs = {}, []

    def worker(t):
        try:
            st = torch.cuda.Stream()
            g = helm.Grid(probs[t][0], 10.0, precision=precision)
            g.set_stream(st.cuda_stream)
            out[t] = [solve(helm, g, probs[t]) for _ in range(2)]
            g.close()
        except Exception as e:  # reported by the main thread
            errs.append(e)

    th = [threading.Thread(target=worker, args=(t,)) for t in range(len(probs))]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errs, errs
    for t, res in out.items():
        for rep, (st, its, U) in enumerate(res):
            assert st == 0, (t, rep, st)
            assert np.array_equal(its, ref[t][1]) and np.array_equal(U, ref[t][2]), (t, rep)
