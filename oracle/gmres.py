"""Restarted, right-preconditioned GMRES in complex128.

Eq. 7 right-preconditions the system: H P^-1 z = f with u = P^-1 z. GMRES
(Saad and Schultz, the method the paper uses) minimises the residual of
that system over the Krylov space. The flexible form keeps
z_j = P^-1 v_j, so the update is u = u0 + Z y. With a fixed P this is
plain right-preconditioned GMRES. A preconditioner that changes from one
step to the next (an inexact V-cycle) is also allowed.

Readings where the paper says nothing: x0 = 0 unless one is given (a warm
start; f = 0 then still returns 0, the unique solution); modified Gram-Schmidt;
complex Givens rotations with a real cosine; stop when the least-squares
residual estimate falls to tol * ||f||, then check the true residual and
restart from the current iterate if it is still above tol.
"""
from __future__ import annotations

import numpy as np

__all__ = ["givens", "arnoldi", "gmres_right", "gmres_split", "block_fgmres"]


def givens(a: complex, b: complex):
    """Rotation (c, s), with c real, that maps (a, b) to (r, 0).

    The rotation is [[c, s], [-conj(s), c]]. Also returns r.
    """
    aa, bb = abs(a), abs(b)
    if aa == 0.0:
        return 0.0, 1.0 + 0j, b
    rho = np.hypot(aa, bb)
    c = aa / rho
    s = (a / aa) * np.conj(b) / rho
    return c, s, (a / aa) * rho


def arnoldi(A, Pinv, v1, m):
    """m steps of Arnoldi with modified Gram-Schmidt on A P^-1.

    Returns V (N x (k+1)), Z (N x k) and Hbar ((k+1) x k), where k <= m is
    the number of steps taken (fewer on breakdown). A Z = V Hbar holds.
    """
    N = v1.shape[0]
    V = np.zeros((N, m + 1), dtype=np.complex128)
    Z = np.zeros((N, m), dtype=np.complex128)
    Hb = np.zeros((m + 1, m), dtype=np.complex128)
    V[:, 0] = v1 / np.linalg.norm(v1)
    for j in range(m):
        Z[:, j] = Pinv(V[:, j])
        w = A(Z[:, j])
        for i in range(j + 1):
            Hb[i, j] = np.vdot(V[:, i], w)
            w = w - Hb[i, j] * V[:, i]
        Hb[j + 1, j] = np.linalg.norm(w)
        if Hb[j + 1, j] == 0.0:
            return V[:, :j + 2], Z[:, :j + 1], Hb[:j + 2, :j + 1]
        V[:, j + 1] = w / Hb[j + 1, j]
    return V, Z, Hb


def gmres_right(A, f, tol, restart, maxiter, Pinv=None, x0=None):
    """Solve A x = f with GMRES(restart), right-preconditioned by Pinv.

    ``A`` and ``Pinv`` are callables on 1D complex128 vectors (Pinv = None
    means no preconditioner). Returns a dict with x, the number of inner
    iterations, restarts, the residual estimate after every iteration
    (relative to ||f||), the true relative residual after every cycle and
    ``converged``.
    """
    f = np.asarray(f, dtype=np.complex128).ravel()
    N = f.shape[0]
    if Pinv is None:
        Pinv = lambda v: v.copy()  # noqa: E731
    x = np.zeros(N, dtype=np.complex128) if x0 is None else np.array(x0, np.complex128).ravel()
    fnorm = np.linalg.norm(f)
    out = {"history": [], "true_residuals": [], "iterations": 0, "restarts": 0,
           "converged": False}
    if fnorm == 0.0:
        # H is non-singular (alpha > 0), so f = 0 has the solution 0 whatever x0 is
        out.update(x=np.zeros(N, dtype=np.complex128), converged=True)
        return out
    its = 0
    while its < maxiter:
        r = f - A(x)
        beta = np.linalg.norm(r)
        if beta <= tol * fnorm:
            out["converged"] = True
            break
        m = restart
        V = np.zeros((N, m + 1), dtype=np.complex128)
        Z = np.zeros((N, m), dtype=np.complex128)
        R = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[:, 0] = r / beta
        k = 0
        for j in range(m):
            Z[:, j] = Pinv(V[:, j])
            w = A(Z[:, j])
            for i in range(j + 1):
                R[i, j] = np.vdot(V[:, i], w)
                w = w - R[i, j] * V[:, i]
            hn = np.linalg.norm(w)
            R[j + 1, j] = hn
            if hn != 0.0:
                V[:, j + 1] = w / hn
            # earlier rotations on the new column
            for i in range(j):
                a, b = R[i, j], R[i + 1, j]
                R[i, j] = cs[i] * a + sn[i] * b
                R[i + 1, j] = -np.conj(sn[i]) * a + cs[i] * b
            cs[j], sn[j], R[j, j] = givens(R[j, j], R[j + 1, j])
            R[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            out["history"].append(abs(g[j + 1]) / fnorm)
            if abs(g[j + 1]) <= tol * fnorm or hn == 0.0 or its >= maxiter:
                break
        # least squares: upper-triangular R[:k,:k] y = g[:k]
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - R[i, i + 1:k] @ y[i + 1:k]) / R[i, i]
        x = x + Z[:, :k] @ y
        out["restarts"] += 1
        rt = np.linalg.norm(f - A(x)) / fnorm
        out["true_residuals"].append(rt)
        if rt <= tol:
            out["converged"] = True
            break
    out["x"] = x
    out["iterations"] = its
    return out


def gmres_split(A, f, tol, restart, maxiter, Ml_inv=None, Mr_inv=None, x0=None):
    """Restarted GMRES on the split-preconditioned system of Eq. 5:

        Ml^-1 A Mr^-1 z = Ml^-1 f,   u = Mr^-1 z.

    The left and right preconditioners are fixed linear maps given by their
    inverses (callables on 1D complex128 vectors; None is the identity).
    Ml = I, Mr = P is Eq. 7. Ml = P, Mr = I is the left-preconditioned
    variant. Over u in x0 + Mr^-1 K_k(Ml^-1 A Mr^-1, r0), each cycle minimises
    the preconditioned residual ||Ml^-1 (f - A u)||_2, with r0 = Ml^-1 (f - A x0).

    Reading (the paper gives no stopping rule for Eq. 5): stop when the
    preconditioned residual falls to tol * ||Ml^-1 f||, the quantity the
    method minimises. With Ml = I that is the true residual test of
    gmres_right. The true relative residual ||f - A u|| / ||f|| is recorded
    after every cycle. Arnoldi uses modified Gram-Schmidt, and the Givens
    rotations have a real cosine, as in gmres_right.
    """
    f = np.asarray(f, dtype=np.complex128).ravel()
    N = f.shape[0]
    ident = lambda v: v.copy()  # noqa: E731
    Ml_inv = ident if Ml_inv is None else Ml_inv
    Mr_inv = ident if Mr_inv is None else Mr_inv
    x = np.zeros(N, dtype=np.complex128) if x0 is None else np.array(x0, np.complex128).ravel()
    fnorm = np.linalg.norm(f)
    out = {"history": [], "true_residuals": [], "iterations": 0, "restarts": 0,
           "converged": False}
    if fnorm == 0.0:
        out.update(x=np.zeros(N, dtype=np.complex128), converged=True)
        return out
    bnorm = np.linalg.norm(Ml_inv(f))
    its = 0
    while its < maxiter:
        r = Ml_inv(f - A(x))
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            out["converged"] = True
            break
        m = restart
        V = np.zeros((N, m + 1), dtype=np.complex128)
        R = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[:, 0] = r / beta
        k = 0
        for j in range(m):
            w = Ml_inv(A(Mr_inv(V[:, j])))
            for i in range(j + 1):
                R[i, j] = np.vdot(V[:, i], w)
                w = w - R[i, j] * V[:, i]
            hn = np.linalg.norm(w)
            R[j + 1, j] = hn
            if hn != 0.0:
                V[:, j + 1] = w / hn
            for i in range(j):
                a, b = R[i, j], R[i + 1, j]
                R[i, j] = cs[i] * a + sn[i] * b
                R[i + 1, j] = -np.conj(sn[i]) * a + cs[i] * b
            cs[j], sn[j], R[j, j] = givens(R[j, j], R[j + 1, j])
            R[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            out["history"].append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or hn == 0.0 or its >= maxiter:
                break
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - R[i, i + 1:k] @ y[i + 1:k]) / R[i, i]
        x = x + Mr_inv(V[:, :k] @ y)
        out["restarts"] += 1
        out["true_residuals"].append(np.linalg.norm(f - A(x)) / fnorm)
        if np.linalg.norm(Ml_inv(f - A(x))) <= tol * bnorm:
            out["converged"] = True
            break
    out["x"] = x
    out["iterations"] = its
    return out


def block_fgmres(A, F, tol, restart, maxiter, Pinv=None):
    """Restarted block flexible GMRES for A X = F with s right-hand sides
    sharing one block Krylov space (right preconditioning as in Eq. 7).

    ``F`` is N x s; ``A`` maps an N x s block to an N x s block; ``Pinv``
    maps one vector (None: identity). Per cycle, from X (0 at first):
    R = F - A X = V_0 B (thin QR); block step j forms Z_j = Pinv(V_j) column
    by column, W = A Z_j, block modified Gram-Schmidt H_ij = V_i^H W,
    W -= V_i H_ij (i <= j), then the thin QR W = V_{j+1} H_{j+1,j}. The
    block Hessenberg least squares min ||E_1 B - Hbar_j Y|| decouples into
    one least-squares problem per column, each column's residual norm is its
    source's residual estimate, and a cycle stops when every estimate is at
    most tol ||F_k|| (or after `restart` block steps); then X += [Z_0 ..
    Z_j] Y and the true residuals decide whether to restart. Returns a dict
    with X, the block steps taken ("iterations"), restarts, the estimate
    history per step (an s-vector each), the true residuals per cycle and
    ``converged``. maxiter bounds the block steps.
    """
    F = np.asarray(F, dtype=np.complex128)
    if F.ndim == 1:
        F = F[:, None]
    N, s = F.shape
    if Pinv is None:
        Pinv = lambda v: v.copy()  # noqa: E731
    fnorm = np.linalg.norm(F, axis=0)
    X = np.zeros_like(F)
    out = {"history": [], "true_residuals": [], "iterations": 0, "restarts": 0,
           "converged": False}
    live = fnorm > 0.0
    its = 0
    while its < maxiter:
        R = F - A(X)
        rn = np.linalg.norm(R, axis=0)
        if np.all(rn[live] <= tol * fnorm[live]):
            out["converged"] = True
            break
        V0, B = np.linalg.qr(R)
        m = restart
        V = [V0]
        Z = []
        Hb = np.zeros(((m + 1) * s, m * s), dtype=np.complex128)
        k = 0
        Y = None
        for j in range(m):
            Zj = np.column_stack([Pinv(V[j][:, c]) for c in range(s)])
            Z.append(Zj)
            W = A(Zj)
            for i in range(j + 1):
                Hij = V[i].conj().T @ W
                Hb[i * s:(i + 1) * s, j * s:(j + 1) * s] = Hij
                W = W - V[i] @ Hij
            Vn, Rn = np.linalg.qr(W)
            Hb[(j + 1) * s:(j + 2) * s, j * s:(j + 1) * s] = Rn
            V.append(Vn)
            its += 1
            k = j + 1
            E = np.zeros(((j + 2) * s, s), dtype=np.complex128)
            E[:s, :] = B
            Hj = Hb[:(j + 2) * s, :(j + 1) * s]
            Y = np.linalg.lstsq(Hj, E, rcond=None)[0]
            est = np.linalg.norm(E - Hj @ Y, axis=0)
            out["history"].append(est / np.where(fnorm > 0, fnorm, 1.0))
            if np.all(est[live] <= tol * fnorm[live]) or its >= maxiter:
                break
        X = X + np.hstack(Z[:k]) @ Y
        out["restarts"] += 1
        tr = np.linalg.norm(F - A(X), axis=0) / np.where(fnorm > 0, fnorm, 1.0)
        out["true_residuals"].append(tr)
        if np.all(tr[live] <= tol):
            out["converged"] = True
            break
    out["X"] = X
    out["iterations"] = its
    return out
