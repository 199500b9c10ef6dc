"""prox of gamma R for R = tau TV_iso + chi_C (Eq. 8), by FGP.

The paper solves this prox with the fast gradient projection (FGP) method of
Beck and Teboulle, "Fast gradient-based algorithms for constrained total
variation image denoising and deblurring problems" (IEEE TIP 2009), cited in
Sec. III-A, without restating it.  This module follows that published
algorithm on the dual variable p = (p_x, p_y):

    x(p)    = P_C(z - lam D^T p)                       lam = gamma * tau
    p_k     = Pi_B(r_k + (1 / (8 lam)) D x(r_k))        (1/(4 d lam) in d dims)
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
    r_{k+1} = p_k + ((t_k - 1) / t_{k+1}) (p_k - p_{k-1})
    output  x(p_K)

with r_1 = p_0 = 0, t_1 = 1.  D is the forward difference with a zero
difference at the last index (Neumann), Pi_B projects each pixel's (p_x, p_y)
onto the unit disk (isotropic TV), and P_C clamps to the box C = [lo, hi].
The paper leaves C as "a bounded convex set" (Sec. II); the box is a reading.
For complex f the reading is a separable prox: Re f and Im f each take this
prox with their own box.

Pinned by: tau = 0 gives the clamp, constant images, the closed-form
two-plateau solution, non-expansiveness and a vanishing duality gap
(tests/test_oracle_prox.py).
"""
from __future__ import annotations

import math

import numpy as np


def grad2(x):
    """Forward differences (D_x x, D_y x), zero at the last column / row."""
    dx = np.zeros_like(x)
    dy = np.zeros_like(x)
    dx[:, :-1] = x[:, 1:] - x[:, :-1]
    dy[:-1, :] = x[1:, :] - x[:-1, :]
    return dx, dy


def grad2_adj(px, py):
    """D^T (p_x, p_y): the exact adjoint of ``grad2``."""
    out = np.zeros_like(px)
    out[:, :-1] -= px[:, :-1]
    out[:, 1:] += px[:, :-1]
    out[:-1, :] -= py[:-1, :]
    out[1:, :] += py[:-1, :]
    return out


def grad3(x):
    """Forward differences (D_x, D_y, D_z) of a [z, y, x] volume, zero at the last index."""
    dx = np.zeros_like(x)
    dy = np.zeros_like(x)
    dz = np.zeros_like(x)
    dx[:, :, :-1] = x[:, :, 1:] - x[:, :, :-1]
    dy[:, :-1, :] = x[:, 1:, :] - x[:, :-1, :]
    dz[:-1, :, :] = x[1:, :, :] - x[:-1, :, :]
    return dx, dy, dz


def grad3_adj(px, py, pz):
    """D^T (p_x, p_y, p_z): the exact adjoint of ``grad3``."""
    out = np.zeros_like(px)
    out[:, :, :-1] -= px[:, :, :-1]
    out[:, :, 1:] += px[:, :, :-1]
    out[:, :-1, :] -= py[:, :-1, :]
    out[:, 1:, :] += py[:, :-1, :]
    out[:-1, :, :] -= pz[:-1, :, :]
    out[1:, :, :] += pz[:-1, :, :]
    return out


def fgp3(z, lam, iters, lo=-np.inf, hi=np.inf):
    """3D FGP (isotropic TV over d = 1..3, the sum of Eq. 8 taken over three
    axes in 3D); dual step 1/(12 lam)."""
    z = np.asarray(z, dtype=np.float64)
    if lam <= 0:
        return np.clip(z, lo, hi)
    pold = [np.zeros_like(z) for _ in range(3)]
    r = [np.zeros_like(z) for _ in range(3)]
    t = 1.0
    step = 1.0 / (12.0 * lam)
    for _ in range(iters):
        x = np.clip(z - lam * grad3_adj(*r), lo, hi)
        d = grad3(x)
        q = [r[i] + step * d[i] for i in range(3)]
        nrm = np.maximum(1.0, np.sqrt(q[0] ** 2 + q[1] ** 2 + q[2] ** 2))
        p = [qi / nrm for qi in q]
        t_new = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        beta = (t - 1.0) / t_new
        r = [p[i] + beta * (p[i] - pold[i]) for i in range(3)]
        pold, t = p, t_new
    return np.clip(z - lam * grad3_adj(*pold), lo, hi)


def tv_iso(x):
    """Isotropic TV: sum_n sqrt(sum_d [D_d x]_n^2) (first term of Eq. 8 without tau)."""
    dx, dy = grad2(x)
    return float(np.sum(np.sqrt(dx * dx + dy * dy)))


def fgp(z, lam, iters, lo=-np.inf, hi=np.inf, return_dual=False):
    """argmin_{x in [lo,hi]} 1/2 ||x - z||^2 + lam TV_iso(x), by ``iters`` FGP steps."""
    z = np.asarray(z, dtype=np.float64)
    if lam <= 0:
        x = np.clip(z, lo, hi)
        return (x, (np.zeros_like(z), np.zeros_like(z))) if return_dual else x
    px_old = np.zeros_like(z)
    py_old = np.zeros_like(z)
    rx = np.zeros_like(z)
    ry = np.zeros_like(z)
    t = 1.0
    step = 1.0 / (8.0 * lam)
    for _ in range(iters):
        x = np.clip(z - lam * grad2_adj(rx, ry), lo, hi)
        dx, dy = grad2(x)
        qx = rx + step * dx
        qy = ry + step * dy
        nrm = np.maximum(1.0, np.sqrt(qx * qx + qy * qy))
        px, py = qx / nrm, qy / nrm
        t_new = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        beta = (t - 1.0) / t_new
        rx = px + beta * (px - px_old)
        ry = py + beta * (py - py_old)
        px_old, py_old, t = px, py, t_new
    x = np.clip(z - lam * grad2_adj(px_old, py_old), lo, hi)
    return (x, (px_old, py_old)) if return_dual else x


def prox_R(z, lam, iters, box_re=(0.0, 2.0), box_im=None):
    """prox of gamma R at z (Eq. 9's outer prox); complex z takes separable Re / Im proxes."""
    z = np.asarray(z)
    fg = fgp3 if z.ndim == 3 else fgp
    xr = fg(z.real, lam, iters, *box_re)
    if box_im is None:
        return xr.astype(np.complex128)
    xi = fg(z.imag, lam, iters, *box_im)
    return xr + 1j * xi


# ---------------------------------------------------------------- anisotropic TV
# R(x) = tau sum_d sum_n |[D_d x]_n| + chi_C, the anisotropic alternative to
# Eq. 8's isotropic TV that Sec. III-A points to (Kamilov, "A parallel
# proximal algorithm for anisotropic total variation minimization", IEEE TIP
# 2017).  Along each axis the differences split into pairs (i, i+1) with i even
# and with i odd; within one parity the pairs are disjoint, so the prox of
# c * sum |x_{i+1} - x_i| over them is closed form: each pair keeps its mean and
# its difference is soft-thresholded by 2c.  With these 2d pieces and the box
# as m = 2d + 1 functions f_j, prox_{sum f_j}(z) is computed by the parallel
# Dykstra-like proximal iteration (Combettes and Pesquet, "Proximal splitting
# methods in signal processing", 2011):
#     z_j <- z                                  for every j
#     repeat:  p_j = prox_{m f_j}(z_j);  x = mean_j p_j;  z_j <- x + z_j - p_j
# Pinned by: convergence to the exact prox computed by an independent dual
# projected-gradient solver, the two-plateau closed form, tau = 0 (clamp),
# constants (tests/test_oracle_prox.py).


def tv_aniso(x):
    """Anisotropic TV: sum over axes and pixels of |forward difference| (zero at the last index)."""
    return float(sum(np.sum(np.abs(np.diff(x, axis=a))) for a in range(x.ndim)))


def pair_shrink(v, axis, parity, c):
    """prox of c * sum_{i = parity mod 2} |v_{i+1} - v_i| along ``axis`` (disjoint pairs)."""
    out = np.array(v, dtype=np.float64, copy=True)
    L = v.shape[axis]
    i0 = np.arange(parity, L - 1, 2)
    a = np.take(v, i0, axis=axis)
    b = np.take(v, i0 + 1, axis=axis)
    mean = 0.5 * (a + b)
    d = b - a
    d = np.sign(d) * np.maximum(np.abs(d) - 2.0 * c, 0.0)
    idx_a = [slice(None)] * v.ndim
    idx_b = [slice(None)] * v.ndim
    idx_a[axis] = i0
    idx_b[axis] = i0 + 1
    out[tuple(idx_a)] = mean - 0.5 * d
    out[tuple(idx_b)] = mean + 0.5 * d
    return out


def ppa_aniso(z, lam, iters, lo=-np.inf, hi=np.inf):
    """argmin_{x in [lo,hi]} 1/2 ||x - z||^2 + lam TV_aniso(x), by ``iters`` parallel proximal iterations."""
    z = np.asarray(z, dtype=np.float64)
    if lam <= 0:
        return np.clip(z, lo, hi)
    pieces = [(a, par) for a in range(z.ndim) for par in (0, 1)]
    m = len(pieces) + 1
    zs = [z.copy() for _ in range(m)]
    x = z.copy()
    for _ in range(iters):
        ps = [pair_shrink(zs[j], a, par, m * lam) for j, (a, par) in enumerate(pieces)]
        ps.append(np.clip(zs[-1], lo, hi))
        x = sum(ps) / m
        zs = [x + zj - pj for zj, pj in zip(zs, ps)]
    return x


def prox_R_aniso(z, lam, iters, box_re=(0.0, 2.0), box_im=None):
    """prox of gamma R with anisotropic TV; complex z takes separable Re / Im proxes."""
    z = np.asarray(z)
    xr = ppa_aniso(z.real, lam, iters, *box_re)
    if box_im is None:
        return xr.astype(np.complex128)
    return xr + 1j * ppa_aniso(z.imag, lam, iters, *box_im)
