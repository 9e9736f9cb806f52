"""The C ABI: the library builds, loads and exports every function that
include/helm.h declares. Runs without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1712_08740_gb300 import helm
    return helm


def declared_functions():
    with open(os.path.join(ROOT, "include", "helm.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(helm_[A-Za-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("helm_create_grid", "helm_set_model", "helm_set_shift", "helm_solve",
                     "helm_solve_batch", "helm_apply_H", "helm_apply_precond", "helm_destroy_grid",
                     "helm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(so, name), name
    assert set(declared_functions()) == set(lib.EXPORTED)


def test_defaults_and_argument_errors_without_gpu(lib):
    o = lib.helm_default_options()
    assert (o.restart, o.precond, o.precision, o.nu1, o.nu2) == (30, 0, 0, 1, 1)
    assert o.omega_jacobi == 0.8 and o.coarse_max == 1500 and o.reorth == 0 and o.graphs == 1
    with pytest.raises(lib.HelmError) as e:
        lib.helm_create_grid(4, (3, 3, 3), 1.0)
    assert e.value.status == 1 and "dim" in e.value.message
    with pytest.raises(lib.HelmError) as e:
        lib.helm_create_grid(2, (1, 5), 1.0)
    assert e.value.status == 1
    with pytest.raises(lib.HelmError):
        lib.helm_create_grid(2, (5, 5), -1.0)


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_1712_08740_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(dirpath, fn)) as fh:
                    src = fh.read()
                assert "oracle" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", src, re.M), fn


def test_solve_footprint_scales(lib):
    o = lib.helm_default_options()
    a = lib.helm_solve_footprint(2, (401, 201), 1, o)
    b = lib.helm_solve_footprint(2, (401, 201), 8, o)
    assert 0 < a < b and b > 8 * 31 * 401 * 201 * 16
    o.precision = 1
    assert lib.helm_solve_footprint(2, (401, 201), 8, o) < b
    assert lib.helm_solve_footprint(0, (401, 201), 8, o) == 0


def test_tile_shape_queries_without_gpu(lib):
    assert lib.helm_num_tile_shapes(1) == 0
    for dim in (2, 3):
        n = lib.helm_num_tile_shapes(dim)
        assert n >= 2
        seen = set()
        for kernel in (0, 1):
            for s in range(n):
                ext, nt = lib.helm_tile_shape(dim, kernel, s)
                rb = lib.helm_tile_rhs_per_block(dim, kernel, s)
                assert nt in (64, 128, 256, 512) and all(e >= 1 for e in ext)
                assert rb in (1, 2, 4) and (dim == 2 or rb == 1)
                if dim == 2:
                    assert ext[2] == 1
                if kernel == 1:                      # up tiles start on even fine nodes
                    assert all(e % 2 == 0 for e in ext[:dim])
                seen.add((kernel, ext, nt, rb))
        assert len(seen) == 2 * n                    # no duplicate shapes
        with pytest.raises(lib.HelmError) as e:
            lib.helm_tile_shape(dim, 0, n)
        assert e.value.status == 1
    with pytest.raises(lib.HelmError):
        lib.helm_tile_shape(2, 2, 0)
    with pytest.raises(lib.HelmError):
        lib.helm_tile_rhs_per_block(2, 0, lib.helm_num_tile_shapes(2))
