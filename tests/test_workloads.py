"""Seeded input generators: deterministic, in range, shaped x-fastest."""
import numpy as np

from workloads import layered_1d, layered_2d, point_sources, request_stream, smooth_random, workload


def test_layered_1d_interfaces():
    c = layered_1d(1001)
    assert c[332] == 1500 and c[333] == 2500 and c[666] == 2500 and c[667] == 3500


def test_smooth_random_seeded_and_in_range():
    a = smooth_random((401, 201), 10.0, seed=0)
    b = smooth_random((401, 201), 10.0, seed=0)
    assert a.shape == (201, 401) and np.array_equal(a, b)
    assert abs(a.min() - 1500) < 1e-9 and abs(a.max() - 4500) < 1e-9
    assert not np.array_equal(a, smooth_random((401, 201), 10.0, seed=1))


def test_layered_2d_range():
    c = layered_2d((81, 41), 7.5, seed=3)
    assert c.shape == (41, 81) and c.min() >= 1500 and c.max() <= 4500
    assert np.all(np.diff(c.mean(axis=1)) >= -150)   # velocity grows with depth on average


def test_point_sources_scaling():
    f = point_sources((5, 4), 2.0, [(1, 2)])
    assert f.shape == (4, 5) and f[2, 1] == 0.25 and np.count_nonzero(f) == 1


def test_workloads_and_stream():
    w = workload("2d_batched")
    assert len(w.sources) == 64 and w.sources[0] == (6, 2) and w.freqs == (5.0, 10.0, 15.0, 20.0)
    reqs = request_stream(50, seed=0)
    t = [r["t_arrival"] for r in reqs]
    assert np.all(np.diff(t) > 0) and all(1 <= len(r["sources"]) <= 8 for r in reqs)
    assert reqs[0]["freq"] == 15.0
