"""The spectrum tool on the library's GPU operators against the oracle's
dense matrices (the paper's Example section, Fig. 2; Eq. 6 and Eq. 7)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import multigrid as mg  # noqa: E402
from oracle import operator as op  # noqa: E402


@pytest.fixture(scope="module")
def spectrum():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1712_08740_gb300 import spectrum as s
    return s


def layered_well(n):
    i = np.arange(n)
    return 1.0 / np.where(i < n // 3, 1500.0, np.where(i < 2 * n // 3, 2500.0, 3500.0))


def nearest_gap(a, b):
    """Largest distance from an eigenvalue of a to the nearest one of b."""
    return float(np.abs(a[:, None] - b[None, :]).min(axis=1).max())


def test_fig2_spectra_and_shift_sweep_1d_well(spectrum):
    """30 Hz, three-layer well, 201 nodes: the GPU operators give the
    oracle's spectra of H and of the exactly preconditioned operator; for the
    shifts (1, 1) and (1, 0.5) the spectrum lies in the disc |lambda - 1/2| <=
    1/2 with positive real parts and the solve converges, while the literal
    sign of Eq. 6, (-1, 1), leaves eigenvalues at negative real parts."""
    from paper_1712_08740_gb300 import helm
    n, h, al = 201, 5.0, 0.01
    om = 2 * np.pi * 30.0
    m = layered_well(n)
    g = helm.Grid((n,), h, precond="exact")
    g.set_model(m, om, al)
    g.set_shift(1.0, 1.0)
    H = op.assemble_H((n,), h, m, om, al).toarray()
    M = op.assemble_M((n,), h, m, om, al, 1.0, 1.0).toarray()
    Hg = spectrum.dense_operator(g, "H")
    assert np.abs(Hg - H).max() <= 1e-13 * np.abs(H).max()
    lam_ref = np.linalg.eigvals(np.linalg.solve(M, H))
    lam = spectrum.eigenvalues(spectrum.dense_operator(g, "preconditioned"))
    assert nearest_gap(lam, lam_ref) < 1e-8 and nearest_gap(lam_ref, lam) < 1e-8
    g.close()

    f = np.zeros(n, complex)
    f[n // 2] = 1.0 / h
    rows = spectrum.shift_sweep((n,), h, m, om, al, [(1.0, 1.0), (1.0, 0.5), (-1.0, 1.0)], f=f)
    by = {r["beta"]: r for r in rows}
    for b in ((1.0, 1.0), (1.0, 0.5)):
        assert by[b]["disc_radius"] <= 0.5 + 1e-9 and by[b]["min_real"] > 0.0
        assert by[b]["status"] == 0 and by[b]["true_rel_residual"] <= 1e-8
    assert by[(-1.0, 1.0)]["min_real"] < -0.1
    lit = op.assemble_M((n,), h, m, om, al, -1.0, 1.0).toarray()
    lam_lit = np.linalg.eigvals(np.linalg.solve(lit, H))
    assert nearest_gap(by[(-1.0, 1.0)]["eigenvalues"], lam_lit) < 1e-8


def test_vcycle_preconditioned_operator_2d(spectrum):
    """With precond="mg" the dense operator is H B, B the V-cycle (three
    levels here): it equals the oracle's H times its V-cycle applied to
    every unit vector."""
    from paper_1712_08740_gb300 import helm
    n, h, al, b, wj = (33, 17), 10.0, 0.01, (1.0, 0.5), 0.8
    om = 2 * np.pi * 10.0
    rng = np.random.default_rng(4)
    m = 1.0 / rng.uniform(1500.0, 4500.0, size=n[::-1])
    g = helm.Grid(n, h, precond="mg", coarse_max=100, omega_jacobi=wj)
    g.set_model(np.ascontiguousarray(m.ravel()), om, al)
    g.set_shift(*b)
    assert g.num_levels == 3
    A = spectrum.dense_operator(g, "preconditioned")
    g.close()
    levels = mg.build_levels(n, h, m, om, al, *b, coarse_max=100)
    N = n[0] * n[1]
    B = np.empty((N, N), complex)
    for i in range(N):
        e = np.zeros(N, complex)
        e[i] = 1.0
        B[:, i] = mg.vcycle(levels, e, 1, 1, wj)
    ref = op.assemble_H(n, h, m, om, al) @ B
    assert np.linalg.norm(A - ref) <= 1e-10 * np.linalg.norm(ref)
    s = spectrum.summarize(spectrum.eigenvalues(A))
    s_ref = spectrum.summarize(np.linalg.eigvals(ref))
    for k in ("min_abs", "max_abs", "disc_radius"):
        assert abs(s[k] - s_ref[k]) <= 1e-8, k
