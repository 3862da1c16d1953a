"""Oracle: preconditioned Krylov solvers in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2.2 / 4.1.5 of the paper: the multigrid V-cycle is used as a
preconditioner of a Krylov method; GMRES uses modified Gram-Schmidt and Givens
rotations (Saad, Iterative Methods for Sparse Linear Systems, Sec. 6.5.3).
CG (Hestenes-Stiefel) and BiCGStab (van der Vorst 1992) are the textbook
algorithms with the preconditioner applied on the right (BiCGStab, GMRES) or
symmetrically (CG).  ``flexible`` CG uses the Polak-Ribiere beta so that a
slightly varying preconditioner (an FP32 V-cycle) is admissible.

Every solver stops when the recursively updated residual satisfies
||r|| <= rtol ||b||, then reports the true residual ||b - A x|| / ||b||.
"""
from __future__ import annotations

import numpy as np


def _result(A, b, x, it, hist):
    nb = np.linalg.norm(b)
    return x, {"iters": it, "true_rel": float(np.linalg.norm(b - A @ x) / nb), "history": hist}


def pcg(A, b, M, rtol=1e-10, maxit=500, flexible=False, x0=None):
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    nb = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / nb]
    if hist[-1] <= rtol:
        return _result(A, b, x, 0, hist)
    z = M(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r_new = r - alpha * q
        hist.append(np.linalg.norm(r_new) / nb)
        if hist[-1] <= rtol:
            return _result(A, b, x, it, hist)
        z_new = M(r_new)
        rz_new = r_new @ z_new
        beta = ((r_new - r) @ z_new) / rz if flexible else rz_new / rz
        p = z_new + beta * p
        r, z, rz = r_new, z_new, rz_new
    return _result(A, b, x, maxit, hist)


def bicgstab(A, b, M, rtol=1e-10, maxit=500, x0=None):
    """Right-preconditioned BiCGStab: solves A M^-1 y = b, x = M^-1 y."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    nb = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / nb]
    if hist[-1] <= rtol:
        return _result(A, b, x, 0, hist)
    rhat = r.copy()
    rho = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, maxit + 1):
        rho_new = rhat @ r
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        phat = M(p)
        v = A @ phat
        alpha = rho_new / (rhat @ v)
        s = r - alpha * v
        if np.linalg.norm(s) / nb <= rtol:
            x = x + alpha * phat
            hist.append(np.linalg.norm(s) / nb)
            return _result(A, b, x, it, hist)
        shat = M(s)
        t = A @ shat
        omega = (t @ s) / (t @ t)
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        rho = rho_new
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= rtol:
            return _result(A, b, x, it, hist)
    return _result(A, b, x, maxit, hist)


def gmres(A, b, M, rtol=1e-10, restart=30, maxit=500, x0=None):
    """Right-preconditioned restarted GMRES with modified Gram-Schmidt and
    Givens rotations.  With a varying preconditioner the stored
    Z_j = M^-1 v_j make it flexible GMRES (Saad 1993)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    nb = np.linalg.norm(b)
    hist = []
    it = 0
    while it < maxit:
        r = b - A @ x
        beta = np.linalg.norm(r)
        hist.append(beta / nb)
        if beta / nb <= rtol:
            break
        m = restart
        V = np.zeros((m + 1, b.size))
        Z = np.zeros((m, b.size))
        Hm = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for j in range(m):
            it += 1
            Z[j] = M(V[j])
            w = A @ Z[j]
            for i in range(j + 1):                     # modified Gram-Schmidt
                Hm[i, j] = w @ V[i]
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] != 0.0:
                V[j + 1] = w / Hm[j + 1, j]
            for i in range(j):                         # apply previous rotations
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            den = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j], sn[j] = Hm[j, j] / den, Hm[j + 1, j] / den
            Hm[j, j] = den
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k_used = j + 1
            hist.append(abs(g[j + 1]) / nb)
            if abs(g[j + 1]) / nb <= rtol or it >= maxit:
                break
        y = np.linalg.solve(np.triu(Hm[:k_used, :k_used]), g[:k_used])
        x = x + Z[:k_used].T @ y
        if hist[-1] <= rtol:
            break
    return _result(A, b, x, it, hist)
