"""Oracle: Krylov methods and the Lanczos condition-number estimate.

Section 4.1 / Section 6: the interface systems are solved by PCG (symmetric
case) or GMRES (strong-scaling tests).  Stopping rule (PETSc default, Table of
tolerances in Section 6): with x0 = 0, stop when the preconditioned residual
norm ||M^-1 r_k|| <= max(rtol ||M^-1 b||, atol); diverged when it exceeds
dtol ||M^-1 b||.  GMRES: restart 30, left preconditioning, modified
Gram-Schmidt (the paper states none of the three; these are PETSc's
defaults).  The condition-number column of Tables 7-8 is read as the ratio
of the extreme eigenvalues of the CG Lanczos tridiagonal matrix.

Pinned by: convergence in n iterations on an n x n SPD system, exact
solutions against numpy.linalg.solve, and the Lanczos estimate against the
eigenvalues of small SPD operators (tests).
"""
from __future__ import annotations

import numpy as np


def pcg(apply_A, apply_M, b, rtol=1e-8, atol=1e-10, dtol=1e4, maxit=1000):
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_M(r)
    zn0 = np.linalg.norm(z)
    alphas, betas = [], []
    info = dict(its=0, reason="atol", alphas=alphas, betas=betas, res0=zn0, res=zn0)
    if zn0 <= atol:
        return x, info
    rz = float(r @ z)
    p = z.copy()
    for k in range(1, maxit + 1):
        q = apply_A(p)
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        z = apply_M(r)
        zn = np.linalg.norm(z)
        alphas.append(alpha)
        info["its"], info["res"] = k, zn
        if zn <= max(rtol * zn0, atol):
            info["reason"] = "converged"
            return x, info
        if zn > dtol * zn0 or not np.isfinite(zn):
            info["reason"] = "diverged"
            return x, info
        rz_new = float(r @ z)
        beta = rz_new / rz
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    info["reason"] = "maxit"
    return x, info


def lanczos_cond(alphas, betas):
    """cond estimate from the CG coefficients (tridiagonal Lanczos matrix)."""
    k = len(alphas)
    if k == 0:
        return 1.0
    T = np.zeros((k, k))
    for i in range(k):
        T[i, i] = 1.0 / alphas[i] + (betas[i - 1] / alphas[i - 1] if i > 0 else 0.0)
        if i + 1 < k:
            T[i, i + 1] = T[i + 1, i] = np.sqrt(betas[i]) / alphas[i]
    ev = np.linalg.eigvalsh(T)
    return float(ev[-1] / ev[0])


def gmres(apply_A, apply_M, b, rtol=1e-8, atol=1e-10, dtol=1e4, maxit=1000, restart=30):
    x = np.zeros_like(b)
    r = apply_M(b)
    beta = np.linalg.norm(r)
    res0 = beta
    info = dict(its=0, reason="atol", res0=res0, res=beta)
    tol = max(rtol * res0, atol)
    if beta <= atol:
        return x, info
    its = 0
    while its < maxit:
        m = restart
        V = np.zeros((m + 1, b.size))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        res = beta
        for j in range(m):
            w = apply_M(apply_A(V[j]))
            for i in range(j + 1):
                H[i, j] = float(w @ V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            res = abs(g[j + 1])
            if res <= tol or its >= maxit or res > dtol * res0:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x += V[:j_done].T @ y
        info["its"], info["res"] = its, res
        if res <= tol:
            info["reason"] = "converged"
            return x, info
        if res > dtol * res0 or not np.isfinite(res):
            info["reason"] = "diverged"
            return x, info
        r = apply_M(b - apply_A(x))
        beta = np.linalg.norm(r)
    info["reason"] = "maxit"
    return x, info
