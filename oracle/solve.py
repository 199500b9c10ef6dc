"""Linear solves of Eq. 13: A u = u_in and A^H v = diag(f)^H H^H w, in FP64.

The paper solves both "by the conjugate gradient method" (Sec. III-A, after
Eq. 13) but A = I - G diag(f) is not Hermitian, so plain CG does not apply.
Reading: any Krylov method that reaches the stated relative residual of the
paper's own system gives the same u up to that residual.  This oracle uses
BiCGSTAB (van der Vorst 1992) and, if that stalls, restarted GMRES (Saad and
Schultz 1986); both stop on the TRUE residual ||b - A x|| / ||b||.  For small
systems ``solve_dense`` is the definition itself (LU of the dense matrix).

Pinned by: dense LU on 16x16 and 24x24 grids (tests/test_oracle_solve.py).
"""
from __future__ import annotations

import numpy as np


def _dot(a, b):
    return np.vdot(a, b)  # conj(a) . b


def bicgstab(apply, b, x0=None, tol=1e-10, maxiter=20000):
    """BiCGSTAB for apply(x) = b; returns (x, iterations, true relative residual)."""
    b = np.asarray(b, dtype=np.complex128).ravel()
    shape_apply = lambda v: apply(v)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).ravel()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    r = b - shape_apply(x)
    rhat = r.copy()
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    while it < maxiter:
        if np.linalg.norm(r) / bn <= tol:
            break
        rho_new = _dot(rhat, r)
        if rho_new == 0:
            break
        beta = (rho_new / rho) * (alpha / omega) if it > 0 else 0.0
        p = r + beta * (p - omega * v)
        v = shape_apply(p)
        alpha = rho_new / _dot(rhat, v)
        s = r - alpha * v
        t = shape_apply(s)
        tt = _dot(t, t).real
        omega = _dot(t, s) / tt if tt > 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        it += 1
    res = np.linalg.norm(b - shape_apply(x)) / bn
    return x, it, res


def gmres(apply, b, x0=None, tol=1e-10, restart=60, maxiter=200):
    """Restarted GMRES(m) with modified Gram-Schmidt and Givens rotations."""
    b = np.asarray(b, dtype=np.complex128).ravel()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).ravel()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    total = 0
    for _ in range(maxiter):
        r = b - apply(x)
        beta = np.linalg.norm(r)
        if beta / bn <= tol:
            break
        V = np.zeros((restart + 1, b.size), dtype=np.complex128)
        Hh = np.zeros((restart + 1, restart), dtype=np.complex128)
        V[0] = r / beta
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        j = 0
        for j in range(restart):
            w = apply(V[j])
            for i in range(j + 1):
                Hh[i, j] = np.vdot(V[i], w)
                w = w - Hh[i, j] * V[i]
            Hh[j + 1, j] = np.linalg.norm(w)
            if Hh[j + 1, j] != 0:
                V[j + 1] = w / Hh[j + 1, j]
            for i in range(j):
                tmp = np.conj(cs[i]) * Hh[i, j] + np.conj(sn[i]) * Hh[i + 1, j]
                Hh[i + 1, j] = -sn[i] * Hh[i, j] + cs[i] * Hh[i + 1, j]
                Hh[i, j] = tmp
            den = np.sqrt(abs(Hh[j, j]) ** 2 + abs(Hh[j + 1, j]) ** 2)
            cs[j] = Hh[j, j] / den
            sn[j] = Hh[j + 1, j] / den
            Hh[j, j] = den
            Hh[j + 1, j] = 0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            total += 1
            if abs(g[j + 1]) / bn <= tol * 0.5:
                break
        k = j + 1
        y = np.linalg.solve(np.triu(Hh[:k, :k]), g[:k])
        x = x + V[:k].T @ y
    res = np.linalg.norm(b - apply(x)) / bn
    return x, total, res


def solve(apply, b, x0=None, tol=1e-10, maxiter=20000):
    """BiCGSTAB, falling back to GMRES(60) from its iterate if it did not reach tol."""
    x, it, res = bicgstab(apply, b, x0, tol, maxiter)
    if res > tol:
        x, it2, res = gmres(apply, b, x, tol)
        it += it2
    return x, it, res


def solve_dense(Amat, b):
    """The definition u = A^{-1} b by dense LU (numpy.linalg.solve)."""
    return np.linalg.solve(Amat, b)


def solve_fields(prob, f, B, x0=None, tol=1e-10, adjoint=False, maxiter=20000):
    """Solve A u_t = B_t (or A^H u_t = B_t) for every transmitter t, one at a time.

    Returns the [T, *f.shape] solutions, iteration counts and true residuals.
    """
    shape = f.shape
    op = prob.AH if adjoint else prob.A
    apply = lambda v: op(f, v.reshape(shape)).ravel()
    out = np.empty_like(np.asarray(B, dtype=np.complex128))
    its, res = [], []
    for t in range(B.shape[0]):
        g = None if x0 is None else x0[t].ravel()
        x, it, r = solve(apply, B[t].ravel(), g, tol, maxiter)
        out[t] = x.reshape(shape)
        its.append(it)
        res.append(r)
    return out, np.array(its), np.array(res)
