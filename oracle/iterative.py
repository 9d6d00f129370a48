"""Iterative refinement with the RS-S factorization as preconditioner.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 5 solves the paper's discretisations to a relative residual of 1e-12
with the approximate factorization as a preconditioner: preconditioned
conjugate gradients for the (real symmetric) Laplace system and GMRES with
restart 20 for the (complex symmetric, indefinite) Lippmann-Schwinger system
(Tables "laplace", "helmholtz" and "h2", column n_it).  The operator A is
applied by FFT (``dense.fft_matvec``) and the preconditioner is
``rss.solve``.  Plain textbook algorithms: CG with a preconditioner M^{-1}
(Hestenes-Stiefel recurrences) and right-preconditioned GMRES(m) (Arnoldi with
modified Gram-Schmidt, Givens rotations for the small least-squares problem).
"""
from __future__ import annotations

import numpy as np


def pcg(apply_A, apply_Minv, b, tol=1e-12, maxit=200):
    """Preconditioned CG from x0 = M^{-1} b; stops when ||b - A x|| <= tol ||b||.
    Returns (x, iterations, relative residual)."""
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    x = apply_Minv(b)
    r = b - apply_A(x)
    it = 0
    rel = np.linalg.norm(r) / nb
    if rel <= tol:
        return x, it, rel
    z = apply_Minv(r)
    p = z.copy()
    rz = np.vdot(r, z).real
    while it < maxit:
        Ap = apply_A(p)
        alpha = rz / np.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        it += 1
        rel = np.linalg.norm(r) / nb
        if rel <= tol:
            break
        z = apply_Minv(r)
        rz_new = np.vdot(r, z).real
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, rel


def gmres(apply_A, apply_Minv, b, tol=1e-12, restart=20, maxit=200):
    """Right-preconditioned GMRES(restart) from x0 = M^{-1} b: solves
    A M^{-1} u = b, x = M^{-1} u.  The iteration count is the number of
    Arnoldi steps.  Returns (x, iterations, relative residual of the true
    residual b - A x)."""
    b = np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b)
    x = apply_Minv(b).astype(np.complex128)
    it = 0
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta / nb <= tol or it >= maxit:
            return x, it, beta / nb
        V = [r / beta]
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        j_done = 0
        for j in range(restart):
            w = apply_A(apply_Minv(V[j]))
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):                           # earlier rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            den = np.sqrt(abs(H[j, j]) ** 2 + abs(H[j + 1, j]) ** 2)
            cs[j] = H[j, j] / den if den else 1.0
            sn[j] = H[j + 1, j] / den if den else 0.0
            H[j, j] = np.conj(cs[j]) * H[j, j] + np.conj(sn[j]) * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            it += 1
            j_done = j + 1
            if abs(g[j + 1]) / nb <= tol or it >= maxit or H[j, j] == 0:
                break
            V.append(w / H[j + 1, j])
        y = np.zeros(j_done, dtype=np.complex128)
        for i in range(j_done - 1, -1, -1):              # back substitution
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]
        u = sum(y[i] * V[i] for i in range(j_done))
        x = x + apply_Minv(u)
