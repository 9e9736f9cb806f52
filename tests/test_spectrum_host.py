"""Host logic of the spectrum tool, on a stand-in grid whose operators are
small numpy matrices (no GPU)."""
import numpy as np
import pytest

pytest.importorskip("torch")


@pytest.fixture(scope="module")
def spectrum():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1712_08740_gb300 import spectrum as s
    return s


class FakeGrid:
    def __init__(self, H, P, M):
        self.H, self.P, self.Mm = H, P, M
        self.N = H.shape[0]

    def apply_H(self, x, y):
        y[:] = self.H @ x

    def apply_precond(self, r, z):
        z[:] = self.P @ r

    def apply_M(self, level, x, y):
        assert level == 0
        y[:] = self.Mm @ x


def test_dense_operator_columns(spectrum):
    rng = np.random.default_rng(1)
    N = 7
    H, P, M = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)) for _ in range(3))
    g = FakeGrid(H, P, M)
    assert np.array_equal(spectrum.dense_operator(g, "H"), H)
    assert np.array_equal(spectrum.dense_operator(g, "M"), M)
    assert np.allclose(spectrum.dense_operator(g, "preconditioned"), H @ P, rtol=0, atol=1e-13)
    with pytest.raises(ValueError):
        spectrum.dense_operator(g, "HM")
    big = FakeGrid(np.zeros((1, 1)), None, None)
    big.N = spectrum.MAX_NODES + 1
    with pytest.raises(ValueError):
        spectrum.dense_operator(big, "H")


def test_summary_of_a_spectrum_on_the_circle(spectrum):
    """lambda = s / (s + j b k^2) for real s > 0 lies on |lambda - 1/2| = 1/2
    (constant k, Dirichlet, no damping): disc radius 1/2, no negative real
    part; its similar matrix D diag(lambda) D^-1 has the same summary."""
    s = np.linspace(0.1, 50.0, 40)
    lam = s / (s + 1j * 0.5 * 10.0)
    out = spectrum.summarize(lam)
    assert abs(out["disc_radius"] - 0.5) < 1e-15
    assert out["negative_real"] == 0.0 and out["min_real"] > 0.0 and out["n"] == 40
    assert out["min_abs"] == pytest.approx(np.abs(lam).min())
    rng = np.random.default_rng(2)
    D = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40)) + 8 * np.eye(40)
    A = D @ np.diag(lam) @ np.linalg.inv(D)
    out2 = spectrum.summarize(spectrum.eigenvalues(A))
    for k in ("disc_radius", "min_abs", "max_abs", "min_real"):
        assert out2[k] == pytest.approx(out[k], abs=1e-9), k
    shifted = spectrum.summarize(np.concatenate([lam, [-0.2 + 0.1j]]))
    assert shifted["negative_real"] == pytest.approx(1 / 41) and shifted["min_real"] == -0.2
