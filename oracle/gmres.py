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

__all__ = ["givens", "arnoldi", "gmres_right", "gmres_split", "block_fgmres", "gcrodr"]


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


def _recycle_space(Ghat, What_Zhat, k):
    """Harmonic Ritz subspace for GCRO-DR: with A Zhat = What Ghat (What with
    orthonormal columns), the harmonic Ritz pairs (theta, p) of A over
    span(Zhat) solve Ghat^H Ghat p = theta Ghat^H (What^H Zhat) p. Returns an
    orthonormal n x k basis P of the eigenvectors of the k smallest |theta|
    (only the span matters) and those theta."""
    A1 = Ghat.conj().T @ Ghat
    A2 = Ghat.conj().T @ What_Zhat
    theta, Y = np.linalg.eig(np.linalg.solve(A2, A1))
    idx = np.argsort(np.abs(theta))[:k]
    P, _ = np.linalg.qr(Y[:, idx])
    return P, theta[idx]


def gcrodr(A, f, tol, restart, k, maxiter, Pinv=None, x0=None, recycle=None):
    """Restarted GMRES with a recycled subspace (GCRO-DR; Parks, de Sturler et
    al.), right-preconditioned as in Eq. 7, for one system of a sequence.

    The recycled space is kept in the preconditioned variable z: Ut (k columns)
    with U = Pinv(Ut) in the solution space and C = A U orthonormal. Arnoldi
    runs on (I - C C^H) A Pinv from a residual orthogonal to C, so the relation
    A [U, Z_m] = [C, V_{m+1}] Ghat with Ghat = [[I, B_m], [0, Hbar_m]] holds;
    each cycle minimises ||r|| over x + span([U, Z_m]) (y_z from the usual
    least squares, y_u = -B_m y_z). After a cycle that did not converge the
    recycled space becomes the k harmonic Ritz vectors of A over
    span([Ut, V_m]) with the smallest |theta| (GMRES-DR in the first cycle,
    when there is no recycled space yet), recombined so that C stays
    orthonormal. Pinv must be a fixed linear map.

    recycle: the Ut (N x k) returned by the previous system of the sequence
    (None: none). For the new operator, U = Pinv(Ut), C = A U is
    orthonormalised (the same column operations on U and Ut), and the initial
    guess gains U C^H r0. Returns a dict with x, iterations, restarts,
    true_residuals, converged and "recycle" (Ut for the next system).
    """
    f = np.asarray(f, dtype=np.complex128).ravel()
    N = f.shape[0]
    if Pinv is None:
        Pinv = lambda v: v.copy()  # noqa: E731
    x = np.zeros(N, dtype=np.complex128) if x0 is None else np.array(x0, np.complex128).ravel()
    fnorm = np.linalg.norm(f)
    out = {"true_residuals": [], "iterations": 0, "restarts": 0, "converged": False, "recycle": None}
    if fnorm == 0.0:
        out.update(x=np.zeros(N, dtype=np.complex128), converged=True, recycle=recycle)
        return out

    def orthonormalise(Ct, U, Ut):
        # thin QR of Ct by modified Gram-Schmidt (twice), the same column
        # operations applied to U and Ut so that A U = C still holds
        Ct, U, Ut = Ct.copy(), U.copy(), Ut.copy()
        kk = Ct.shape[1]
        for i in range(kk):
            for _ in range(2):
                for l in range(i):
                    c = np.vdot(Ct[:, l], Ct[:, i])
                    Ct[:, i] -= c * Ct[:, l]
                    U[:, i] -= c * U[:, l]
                    Ut[:, i] -= c * Ut[:, l]
            nrm = np.linalg.norm(Ct[:, i])
            Ct[:, i] /= nrm
            U[:, i] /= nrm
            Ut[:, i] /= nrm
        return Ct, U, Ut

    r = f - A(x)
    C = U = Ut = None
    if recycle is not None and recycle.shape[1] > 0:
        Ut = np.array(recycle, dtype=np.complex128)
        U = np.column_stack([Pinv(Ut[:, i]) for i in range(Ut.shape[1])])
        Ct = np.column_stack([A(U[:, i]) for i in range(U.shape[1])])
        C, U, Ut = orthonormalise(Ct, U, Ut)
        c = C.conj().T @ r
        x = x + U @ c
        r = r - C @ c
    its = 0
    while its < maxiter:
        beta = np.linalg.norm(r)
        if beta <= tol * fnorm:
            out["converged"] = True
            break
        kc = 0 if C is None else C.shape[1]
        m = restart
        V = np.zeros((N, m + 1), dtype=np.complex128)
        Z = np.zeros((N, m), dtype=np.complex128)
        Hb = np.zeros((m + 1, m), dtype=np.complex128)
        B = np.zeros((kc, m), dtype=np.complex128)
        V[:, 0] = r / beta
        steps = 0
        y = None
        for j in range(m):
            Z[:, j] = Pinv(V[:, j])
            w = A(Z[:, j])
            if kc:
                B[:, j] = C.conj().T @ w
                w = w - C @ B[:, j]
            for i in range(j + 1):
                Hb[i, j] = np.vdot(V[:, i], w)
                w = w - Hb[i, j] * V[:, i]
            Hb[j + 1, j] = np.linalg.norm(w)
            V[:, j + 1] = w / Hb[j + 1, j]
            its += 1
            steps = j + 1
            e1 = np.zeros(j + 2, dtype=np.complex128)
            e1[0] = beta
            y = np.linalg.lstsq(Hb[:j + 2, :j + 1], e1, rcond=None)[0]
            est = np.linalg.norm(e1 - Hb[:j + 2, :j + 1] @ y)
            if est <= tol * fnorm or its >= maxiter:
                break
        x = x + Z[:, :steps] @ y
        if kc:
            x = x - U @ (B[:, :steps] @ y)
        r = f - A(x)
        out["restarts"] += 1
        out["true_residuals"].append(np.linalg.norm(r) / fnorm)
        if np.linalg.norm(r) <= tol * fnorm:
            out["converged"] = True
            break
        if k > 0 and steps == m:
            # harmonic Ritz vectors over span([Ut, V_m]) (z variable) and their
            # images: Zhat = [U, Z_m] (solution), What = [C, V_{m+1}]
            n = kc + m
            Ghat = np.zeros((n + 1, n), dtype=np.complex128)
            Ghat[:kc, :kc] = np.eye(kc)
            Ghat[:kc, kc:] = B
            Ghat[kc:, kc:] = Hb
            Wt = np.zeros((n + 1, n), dtype=np.complex128)   # What^H [Ut, V_m]
            if kc:
                Wt[:kc, :kc] = C.conj().T @ Ut
                Wt[kc:, :kc] = V.conj().T @ Ut
            Wt[kc:kc + m, kc:] = np.eye(m)
            P, _ = _recycle_space(Ghat, Wt, min(k, n))
            Zz = np.hstack([Ut, V[:, :m]]) if kc else V[:, :m]
            Zu = np.hstack([U, Z]) if kc else Z
            Wh = np.hstack([C, V]) if kc else V
            Q = Ghat @ P
            # C = What Q R^-1 with R from Q^H Q (What has orthonormal columns)
            R = np.linalg.cholesky(Q.conj().T @ Q).conj().T
            Rinv = np.linalg.inv(R)
            C = Wh @ (Q @ Rinv)
            U = Zu @ (P @ Rinv)
            Ut = Zz @ (P @ Rinv)
            c = C.conj().T @ r
            x = x + U @ c
            r = r - C @ c
    out["x"] = x
    out["iterations"] = its
    out["recycle"] = Ut
    out["U"], out["C"] = U, C
    return out
