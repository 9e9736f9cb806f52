"""ctypes binding of libhelm (include/helm.h): argument marshalling only.

Every function here takes the C function's name and arguments. Arrays may
be torch tensors (CUDA or CPU) or numpy arrays, complex128 (or float64 for
the slowness), C-contiguous; their raw pointers go straight to the library,
which reads host or device memory as the pointer says. All arithmetic runs
in the library's CUDA kernels. If the shared library is missing this module
raises at import: there is no other code path.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libhelm.so")

HELM_OK = 0
STATUS_NAMES = {0: "HELM_OK", 1: "HELM_ERR_ARG", 2: "HELM_ERR_NOMEM", 3: "HELM_ERR_CUDA",
                4: "HELM_ERR_NOT_CONVERGED", 5: "HELM_ERR_BREAKDOWN", 6: "HELM_ERR_NONFINITE",
                7: "HELM_ERR_STATE", 8: "HELM_ERR_UNSUPPORTED"}
PRECOND = {"mg": 0, "exact": 1, "none": 2}
PRECISION = {"f64": 0, "mixed": 1, "mixed_ds": 2, "mixed_c64": 3}
SIDE = {"right": 0, "left": 1, "split": 2}

EXPORTED = ("helm_default_options", "helm_create_grid", "helm_destroy_grid", "helm_set_stream",
            "helm_set_options", "helm_get_options", "helm_set_model", "helm_set_shift",
            "helm_solve", "helm_solve_batch", "helm_solve_batch_warm", "helm_apply_H", "helm_apply_H_ds", "helm_apply_M",
            "helm_apply_precond", "helm_true_residual", "helm_num_levels", "helm_level_info",
            "helm_last_error", "helm_kernel_launches", "helm_profile_start", "helm_profile_stop",
            "helm_time_kernel", "helm_true_residual_noalloc", "helm_solve_footprint",
            "helm_server_create", "helm_server_submit", "helm_server_wait", "helm_server_poll",
            "helm_server_clock", "helm_server_destroy", "helm_num_tile_shapes", "helm_tile_shape",
            "helm_tile_rhs_per_block",
            "helm_set_tiles", "helm_get_tiles", "helm_autotune", "helm_set_wait_limit_ns",
            "helm_set_density", "helm_block_gram", "helm_block_combine")


class helm_options(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_iters", ctypes.c_int), ("precond", ctypes.c_int),
                ("precision", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("omega_jacobi", ctypes.c_double), ("coarse_max", ctypes.c_int),
                ("reorth", ctypes.c_int), ("graphs", ctypes.c_int), ("side", ctypes.c_int),
                ("block", ctypes.c_int), ("recycle", ctypes.c_int)]


class helm_server_config(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int), ("memory_budget", ctypes.c_size_t),
                ("options", helm_options), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("coalesce", ctypes.c_int)]


class helm_request(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("h", ctypes.c_double),
                ("m", ctypes.c_void_p), ("omega", ctypes.c_double), ("alpha", ctypes.c_double),
                ("nrhs", ctypes.c_int), ("f", ctypes.c_void_p), ("tol", ctypes.c_double)]


class helm_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int), ("nrhs", ctypes.c_int),
                ("iterations_max", ctypes.c_int), ("true_rel_residual_max", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("footprint_bytes", ctypes.c_size_t)]


HELM_TUNE_TILES, HELM_TUNE_SMOOTHER = 1, 2
HELM_TUNE_MAX_LEVELS, HELM_TUNE_MAX_NU = 16, 4


class helm_tune_report(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int),
                ("down_shape", ctypes.c_int * HELM_TUNE_MAX_LEVELS),
                ("up_shape", ctypes.c_int * HELM_TUNE_MAX_LEVELS),
                ("down_us", ctypes.c_double * HELM_TUNE_MAX_LEVELS),
                ("up_us", ctypes.c_double * HELM_TUNE_MAX_LEVELS),
                ("down_default_us", ctypes.c_double * HELM_TUNE_MAX_LEVELS),
                ("up_default_us", ctypes.c_double * HELM_TUNE_MAX_LEVELS),
                ("n_nu", ctypes.c_int),
                ("nu", (ctypes.c_int * 2) * HELM_TUNE_MAX_NU),
                ("nu_ms", ctypes.c_double * HELM_TUNE_MAX_NU),
                ("nu_iterations", ctypes.c_int * HELM_TUNE_MAX_NU),
                ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int)]


class HelmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhelm.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "helm_default_options": (None, [ctypes.POINTER(helm_options)]),
        "helm_create_grid": (I, [I, ctypes.POINTER(ctypes.c_int64), D, ctypes.POINTER(P)]),
        "helm_destroy_grid": (None, [P]),
        "helm_set_stream": (I, [P, P]),
        "helm_set_options": (I, [P, ctypes.POINTER(helm_options)]),
        "helm_get_options": (I, [P, ctypes.POINTER(helm_options)]),
        "helm_set_model": (I, [P, P, D, D]),
        "helm_set_shift": (I, [P, D, D]),
        "helm_set_density": (I, [P, P]),
        "helm_block_gram": (I, [I, I, ctypes.c_size_t, ctypes.c_size_t, P, P, P]),
        "helm_block_combine": (I, [I, I, ctypes.c_size_t, ctypes.c_size_t, P, P, ctypes.c_float, P]),
        "helm_solve": (I, [P, P, D, P, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "helm_solve_batch": (I, [P, I, P, D, P, P, P]),
        "helm_solve_batch_warm": (I, [P, I, P, D, P, P, P]),
        "helm_apply_H": (I, [P, P, P]),
        "helm_apply_H_ds": (I, [P, P, P]),
        "helm_apply_M": (I, [P, I, P, P]),
        "helm_apply_precond": (I, [P, P, P]),
        "helm_true_residual": (I, [P, P, P, ctypes.POINTER(D)]),
        "helm_num_levels": (I, [P]),
        "helm_level_info": (I, [P, I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(D)]),
        "helm_last_error": (ctypes.c_char_p, []),
        "helm_kernel_launches": (ctypes.c_uint64, []),
        "helm_set_wait_limit_ns": (I, [ctypes.c_uint64]),
        "helm_profile_start": (I, []),
        "helm_profile_stop": (I, [ctypes.c_char_p, ctypes.c_size_t]),
        "helm_time_kernel": (I, [P, ctypes.c_char_p, I, I, ctypes.POINTER(D), ctypes.POINTER(D),
                                 ctypes.POINTER(D)]),
        "helm_true_residual_noalloc": (I, [P, I, P, P, P]),
        "helm_solve_footprint": (ctypes.c_size_t, [I, ctypes.POINTER(ctypes.c_int64), I,
                                                   ctypes.POINTER(helm_options)]),
        "helm_server_create": (I, [ctypes.POINTER(helm_server_config), ctypes.POINTER(P)]),
        "helm_server_submit": (I, [P, ctypes.POINTER(helm_request), P,
                                   ctypes.POINTER(ctypes.c_uint64)]),
        "helm_server_wait": (I, [P, ctypes.c_uint64, ctypes.POINTER(helm_result)]),
        "helm_server_poll": (I, [P, ctypes.c_uint64, ctypes.POINTER(I)]),
        "helm_server_clock": (D, [P]),
        "helm_server_destroy": (None, [P]),
        "helm_num_tile_shapes": (I, [I]),
        "helm_tile_shape": (I, [I, I, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "helm_tile_rhs_per_block": (I, [I, I, I, ctypes.POINTER(I)]),
        "helm_set_tiles": (I, [P, I, I, I]),
        "helm_get_tiles": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "helm_autotune": (I, [P, I, P, D, I, ctypes.POINTER(helm_tune_report)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


# Grids and servers still open at interpreter exit are closed by an atexit
# hook, while the CUDA runtime is still up: left to the garbage collector they
# would free device memory during interpreter teardown, after the runtime may
# have begun unloading.
_live = weakref.WeakSet()


def _close_live():
    for obj in list(_live):
        try:
            obj.close()
        except Exception:
            pass


atexit.register(_close_live)


def _check(status):
    if status != HELM_OK:
        raise HelmError(status, _lib.helm_last_error().decode())


def _ptr(a, dtype):
    """Raw pointer of a contiguous torch tensor or numpy array of `dtype`."""
    if hasattr(a, "data_ptr"):                  # torch.Tensor
        import torch
        want = {np.complex128: torch.complex128, np.float64: torch.float64}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous numpy {np.dtype(dtype).name} array")
    return ctypes.c_void_p(a.ctypes.data)


# ------------------------------------------------------------------ C functions, same names

def helm_default_options():
    o = helm_options()
    _lib.helm_default_options(ctypes.byref(o))
    return o


def helm_create_grid(dim, n, h):
    nn = (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    g = ctypes.c_void_p()
    _check(_lib.helm_create_grid(int(dim), nn, float(h), ctypes.byref(g)))
    return g


def helm_destroy_grid(g):
    _lib.helm_destroy_grid(g)


def helm_set_stream(g, stream):
    _check(_lib.helm_set_stream(g, ctypes.c_void_p(int(stream))))


def helm_set_options(g, opt):
    _check(_lib.helm_set_options(g, ctypes.byref(opt)))


def helm_get_options(g):
    o = helm_options()
    _check(_lib.helm_get_options(g, ctypes.byref(o)))
    return o


def helm_set_model(g, m, omega, alpha):
    _check(_lib.helm_set_model(g, _ptr(m, np.float64), float(omega), float(alpha)))


def helm_set_density(g, rho):
    """rho of Eq. 1 per node (None: constant density)."""
    _check(_lib.helm_set_density(g, None if rho is None else _ptr(rho, np.float64)))


def helm_set_shift(g, beta1, beta2):
    _check(_lib.helm_set_shift(g, float(beta1), float(beta2)))


def helm_solve(g, f, tol, u, check=True):
    """Returns (status, iterations, true relative residual); raises unless
    check is False."""
    its = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = _lib.helm_solve(g, _ptr(f, np.complex128), float(tol), _ptr(u, np.complex128),
                         ctypes.byref(its), ctypes.byref(rel))
    if check:
        _check(st)
    return st, its.value, rel.value


def helm_solve_batch(g, nrhs, f, tol, u, check=True, warm=False):
    """warm=True: u holds the initial guess on entry (helm_solve_batch_warm)."""
    its = np.zeros(nrhs, dtype=np.int32)
    rel = np.zeros(nrhs, dtype=np.float64)
    fn = _lib.helm_solve_batch_warm if warm else _lib.helm_solve_batch
    st = fn(g, int(nrhs), _ptr(f, np.complex128), float(tol), _ptr(u, np.complex128),
            its.ctypes.data_as(ctypes.c_void_p), rel.ctypes.data_as(ctypes.c_void_p))
    if check:
        _check(st)
    return st, its, rel


def helm_apply_H(g, x, y):
    _check(_lib.helm_apply_H(g, _ptr(x, np.complex128), _ptr(y, np.complex128)))


def helm_apply_H_ds(g, x, y):
    _check(_lib.helm_apply_H_ds(g, _ptr(x, np.complex128), _ptr(y, np.complex128)))


def helm_apply_M(g, level, x, y):
    _check(_lib.helm_apply_M(g, int(level), _ptr(x, np.complex128), _ptr(y, np.complex128)))


def helm_apply_precond(g, r, z):
    _check(_lib.helm_apply_precond(g, _ptr(r, np.complex128), _ptr(z, np.complex128)))


def helm_true_residual(g, f, u):
    rel = ctypes.c_double(0.0)
    _check(_lib.helm_true_residual(g, _ptr(f, np.complex128), _ptr(u, np.complex128),
                                   ctypes.byref(rel)))
    return rel.value


def helm_true_residual_noalloc(g, nrhs, f, u):
    """Relative residuals of nrhs device-resident pairs (f_k, u_k), computed by
    the library without allocating device memory (see include/helm.h).
    ``g`` is a Grid: its node count bounds what f and u must hold."""
    N = g.N
    for name, a in (("f", f), ("u", u)):
        size = a.numel() if hasattr(a, "numel") else np.size(a)
        if size < int(nrhs) * N:
            raise ValueError(f"{name} holds {size} values, fewer than nrhs * N = {int(nrhs) * N}")
    rel = np.zeros(int(nrhs), dtype=np.float64)
    _check(_lib.helm_true_residual_noalloc(g._g, int(nrhs), _ptr(f, np.complex128),
                                           _ptr(u, np.complex128),
                                           rel.ctypes.data_as(ctypes.c_void_p)))
    return rel


def helm_num_levels(g):
    return int(_lib.helm_num_levels(g))


def helm_level_info(g, level):
    nn = (ctypes.c_int64 * 3)()
    h = ctypes.c_double(0.0)
    _check(_lib.helm_level_info(g, int(level), nn, ctypes.byref(h)))
    return tuple(int(v) for v in nn), h.value


def helm_last_error():
    return _lib.helm_last_error().decode()


def helm_set_wait_limit_ns(ns):
    """Time limit of the streamed double-single kernels' copy waits (0: default)."""
    _check(_lib.helm_set_wait_limit_ns(int(ns)))


def _ptr_c64(a):
    """Raw pointer of a contiguous complex64 torch tensor."""
    import torch
    if a.dtype != torch.complex64 or not a.is_contiguous() or not a.is_cuda:
        raise TypeError("expected a contiguous complex64 CUDA tensor")
    return ctypes.c_void_p(a.data_ptr())


def helm_block_gram(V, W, N):
    """G = V^H W on the tensor cores; V (nv x ld), W (s x ld) complex64 CUDA
    tensors with zeros beyond column N. Returns G as an (nv, s) complex128 array."""
    nv, ld = V.shape
    s = W.shape[0]
    G = np.zeros((nv, s), dtype=np.complex128)
    _check(_lib.helm_block_gram(int(nv), int(s), int(N), int(ld), _ptr_c64(V), _ptr_c64(W),
                                G.ctypes.data_as(ctypes.c_void_p)))
    return G


def helm_block_combine(V, C, alpha, W, N):
    """W = alpha W + C^T-combination: W_c = alpha W_c + sum_i V_i C[i, c] (in place)."""
    nv, ld = V.shape
    s = W.shape[0]
    C = np.ascontiguousarray(C, dtype=np.complex128)
    _check(_lib.helm_block_combine(int(nv), int(s), int(N), int(ld), _ptr_c64(V),
                                   C.ctypes.data_as(ctypes.c_void_p), float(alpha), _ptr_c64(W)))


def helm_kernel_launches():
    return int(_lib.helm_kernel_launches())


def helm_profile_start():
    _check(_lib.helm_profile_start())


def helm_profile_stop():
    """Per-kernel {name: {launches, ms, bytes, flops64}} since helm_profile_start."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    _check(_lib.helm_profile_stop(buf, len(buf)))
    return json.loads(buf.value.decode())


def helm_time_kernel(g, kernel, j, reps):
    """(microseconds per launch, algorithmic bytes, FP64 flops) of one kernel."""
    us, b, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.helm_time_kernel(g, kernel.encode(), int(j), int(reps), ctypes.byref(us),
                                 ctypes.byref(b), ctypes.byref(fl)))
    return us.value, b.value, fl.value


def helm_num_tile_shapes(dim):
    return _lib.helm_num_tile_shapes(int(dim))


def helm_tile_shape(dim, kernel, shape):
    """((sx, sy, sz), threads) of a fused-kernel tile shape; kernel 0 = down, 1 = up."""
    ext, nt = (ctypes.c_int * 3)(), ctypes.c_int()
    _check(_lib.helm_tile_shape(int(dim), int(kernel), int(shape), ext, ctypes.byref(nt)))
    return tuple(ext), nt.value


def helm_tile_rhs_per_block(dim, kernel, shape):
    """Right-hand sides one block of a fused-kernel tile shape computes."""
    rb = ctypes.c_int()
    _check(_lib.helm_tile_rhs_per_block(int(dim), int(kernel), int(shape), ctypes.byref(rb)))
    return rb.value


def helm_set_tiles(g, level, down_shape, up_shape):
    _check(_lib.helm_set_tiles(g, int(level), int(down_shape), int(up_shape)))


def helm_get_tiles(g, level):
    d, u = ctypes.c_int(), ctypes.c_int()
    _check(_lib.helm_get_tiles(g, int(level), ctypes.byref(d), ctypes.byref(u)))
    return d.value, u.value


def helm_autotune(g, nrhs, f, tol, flags):
    """Runs the autotuner; returns its report as a dict."""
    rep = helm_tune_report()
    fp = _ptr(f, np.complex128) if f is not None else None
    _check(_lib.helm_autotune(g, int(nrhs), fp, float(tol), int(flags), ctypes.byref(rep)))
    L = rep.levels
    return {
        "levels": L,
        "down_shape": list(rep.down_shape[:L]), "up_shape": list(rep.up_shape[:L]),
        "down_us": list(rep.down_us[:L]), "up_us": list(rep.up_us[:L]),
        "down_default_us": list(rep.down_default_us[:L]),
        "up_default_us": list(rep.up_default_us[:L]),
        "nu_candidates": [tuple(rep.nu[k]) for k in range(rep.n_nu)],
        "nu_ms": list(rep.nu_ms[:rep.n_nu]), "nu_iterations": list(rep.nu_iterations[:rep.n_nu]),
        "nu1": rep.nu1, "nu2": rep.nu2,
    }


# ------------------------------------------------------------------ convenience wrapper

class Grid:
    """Owns one helm_grid. ``n`` is the node count per axis, x first."""

    def __init__(self, n, h, *, restart=30, precond="mg", precision="f64", nu1=1, nu2=1,
                 omega_jacobi=0.8, coarse_max=1500, reorth=0, max_iters=5000, graphs=True,
                 side="right", block=False, recycle=0):
        self.n = tuple(int(k) for k in n)
        self.N = int(np.prod(self.n))
        self.h = float(h)
        self._g = helm_create_grid(len(self.n), self.n, h)
        _live.add(self)
        self.set_options(restart=restart, precond=precond, precision=precision, nu1=nu1,
                         nu2=nu2, omega_jacobi=omega_jacobi, coarse_max=coarse_max,
                         reorth=reorth, max_iters=max_iters, graphs=graphs, side=side, block=block,
                         recycle=recycle)

    def set_options(self, **kw):
        o = helm_get_options(self._g)
        for k, v in kw.items():
            if k == "precond":
                v = PRECOND[v]
            elif k == "precision":
                v = PRECISION[v]
            elif k == "graphs":
                v = int(bool(v))
            elif k == "reorth":
                v = int(v)
            elif k == "side":
                v = SIDE[v]
            elif k == "block":
                v = int(bool(v))
            setattr(o, k, v)
        helm_set_options(self._g, o)

    def set_model(self, m, omega, alpha):
        helm_set_model(self._g, m, omega, alpha)

    def set_shift(self, beta1, beta2):
        helm_set_shift(self._g, beta1, beta2)

    def set_density(self, rho):
        helm_set_density(self._g, rho)

    def set_stream(self, stream):
        helm_set_stream(self._g, stream)

    def solve(self, f, tol, u, check=True, warm=False):
        """warm=True: start from the initial guess that u holds."""
        if warm:
            st, its, rel = helm_solve_batch(self._g, 1, f, tol, u, check, warm=True)
            return st, int(its[0]), float(rel[0])
        return helm_solve(self._g, f, tol, u, check)

    def solve_batch(self, nrhs, f, tol, u, check=True, warm=False):
        return helm_solve_batch(self._g, nrhs, f, tol, u, check, warm)

    def apply_H(self, x, y):
        helm_apply_H(self._g, x, y)

    def apply_H_ds(self, x, y):
        helm_apply_H_ds(self._g, x, y)

    def apply_M(self, level, x, y):
        helm_apply_M(self._g, level, x, y)

    def apply_precond(self, r, z):
        helm_apply_precond(self._g, r, z)

    def true_residual(self, f, u):
        return helm_true_residual(self._g, f, u)

    def time_kernel(self, kernel, j, reps=50):
        return helm_time_kernel(self._g, kernel, j, reps)

    def autotune(self, nrhs, f, tol, tiles=True, smoother=True):
        flags = (HELM_TUNE_TILES if tiles else 0) | (HELM_TUNE_SMOOTHER if smoother else 0)
        return helm_autotune(self._g, nrhs, f, tol, flags)

    def set_tiles(self, level, down_shape, up_shape):
        helm_set_tiles(self._g, level, down_shape, up_shape)

    def get_tiles(self, level):
        return helm_get_tiles(self._g, level)

    @property
    def num_levels(self):
        return helm_num_levels(self._g)

    def level_info(self, level):
        return helm_level_info(self._g, level)

    def close(self):
        if self._g:
            helm_destroy_grid(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving

def helm_solve_footprint(dim, n, nrhs, opt):
    nn = (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    return int(_lib.helm_solve_footprint(int(dim), nn, int(nrhs), ctypes.byref(opt)))


def helm_server_create(cfg):
    s = ctypes.c_void_p()
    _check(_lib.helm_server_create(ctypes.byref(cfg), ctypes.byref(s)))
    return s


def helm_server_submit(s, req, u):
    rid = ctypes.c_uint64(0)
    _check(_lib.helm_server_submit(s, ctypes.byref(req), _ptr(u, np.complex128), ctypes.byref(rid)))
    return rid.value


def helm_server_wait(s, rid, check=True):
    res = helm_result()
    st = _lib.helm_server_wait(s, ctypes.c_uint64(rid), ctypes.byref(res))
    if check:
        _check(st)
    return st, res


def helm_server_poll(s, rid):
    d = ctypes.c_int(0)
    _check(_lib.helm_server_poll(s, ctypes.c_uint64(rid), ctypes.byref(d)))
    return bool(d.value)


def helm_server_clock(s):
    return float(_lib.helm_server_clock(s))


def helm_server_destroy(s):
    _lib.helm_server_destroy(s)


class Server:
    """Request loop on the current CUDA device (see include/helm.h, serving)."""

    def __init__(self, workers=4, memory_budget=64 << 30, beta=(1.0, 0.5), coalesce=0, **opts):
        o = helm_default_options()
        for k, v in opts.items():
            if k == "precond":
                v = PRECOND[v]
            elif k == "precision":
                v = PRECISION[v]
            setattr(o, k, int(v) if k != "omega_jacobi" else float(v))
        self.options = o
        cfg = helm_server_config(int(workers), int(memory_budget), o, float(beta[0]), float(beta[1]),
                                 int(coalesce))
        self._s = helm_server_create(cfg)
        self._keep = {}
        _live.add(self)

    def submit(self, n, h, m, omega, alpha, f, tol):
        """Queues one request; f is (nrhs, N) complex128, m (N,) float64 (host)."""
        n = tuple(int(k) for k in n)
        N = int(np.prod(n))
        m = np.ascontiguousarray(np.asarray(m, dtype=np.float64).ravel())
        f = np.ascontiguousarray(np.asarray(f, dtype=np.complex128).reshape(-1, N))
        u = np.zeros_like(f)
        req = helm_request(len(n), (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n)))),
                           float(h), ctypes.c_void_p(m.ctypes.data), float(omega), float(alpha),
                           int(f.shape[0]), ctypes.c_void_p(f.ctypes.data), float(tol))
        rid = helm_server_submit(self._s, req, u)
        self._keep[rid] = (m, f, u)
        return rid

    def wait(self, rid, check=True):
        st, res = helm_server_wait(self._s, rid, check=check)
        _, _, u = self._keep.pop(rid)
        return st, res, u

    def done(self, rid):
        return helm_server_poll(self._s, rid)

    def clock(self):
        return helm_server_clock(self._s)

    def close(self):
        if self._s:
            helm_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
