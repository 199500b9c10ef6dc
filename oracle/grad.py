"""Data term D (Eq. 7) and its gradient by the adjoint-state method (Prop. 1).

For every transmitter t (the experiments sum D over transmitters, Sec. IV):
    u_t = A^{-1} u_in,t                        (Eq. 13, left)
    w_t = H diag(u_t) f - y_t = Z(f) - y_t     (Eq. 5, Prop. 1)
    D   = 1/2 sum_t ||w_t||^2                  (Eq. 7)
    z_t = H^H w_t
    v_t = A^{-H} diag(f)^H z_t                 (Eq. 13, right)
    g  += conj(u_t) * (z_t + G^H v_t)          (Eq. 12 before taking Re)
grad D = Re g for real f (Eq. 12).  For complex f (absorbing objects, outside
the paper's real-f assumption) the reading is: (Re f, Im f) are independent
real unknowns, dD/dRe f = Re g, dD/dIm f = Im g, with A^H = I - diag(conj f) G^H.

Receiver masks (a transmitter records only some receivers, as in the Fresnel
experiments of Sec. IV): with mask[t, m] in {0, 1}, w_t = mask_t (Z_t - y_t), so
D and g only see active receivers.

Pinned by: central finite differences of D, the Taylor-remainder slope, the
f = 0 special case, and brute-force dense solves (tests/test_oracle_grad.py);
masks by per-transmitter sub-problems holding only the active receivers
(tests/test_oracle_fresnel.py).
"""
from __future__ import annotations

import numpy as np

from .model import conv_G
from .solve import solve_fields


def forward(prob, f, tol=1e-10, x0=None):
    """Total fields u_t (Eq. 13) and clean measurements Z_t = H diag(u_t) f (Eq. 5)."""
    u, its, res = solve_fields(prob, f, prob.u_in, x0=x0, tol=tol)
    return u, prob.sense(f, u), its, res


def data_and_grad(prob, f, y, tol=1e-10, u0=None, v0=None, return_fields=False, mask=None):
    """D(f) and the complex vector g of Prop. 1 (grad D = Re g for real f)."""
    n = prob.n
    u, Z, _, _ = forward(prob, f, tol, x0=u0)
    w = Z - y
    if mask is not None:
        w = w * np.asarray(mask, dtype=np.float64)
    D = 0.5 * float(np.sum(np.abs(w) ** 2))
    z = (w @ np.conj(prob.H)).reshape((-1,) + f.shape)  # H^H w_t for each t
    b = np.conj(f)[None] * z
    v, _, _ = solve_fields(prob, f, b, x0=v0, tol=tol, adjoint=True)
    g = np.zeros(f.shape, dtype=np.complex128)
    for t in range(prob.T):
        g += np.conj(u[t]) * (z[t] + conv_G(v[t], prob.ghat, n, adjoint=True))
    if return_fields:
        return D, g, u, v
    return D, g


def data_term(prob, f, y, tol=1e-12, mask=None):
    """D(f) = 1/2 sum_t ||y_t - Z_t(f)||^2 (Eq. 7), over active receivers if masked."""
    _, Z, _, _ = forward(prob, f, tol)
    w = Z - y if mask is None else (Z - y) * np.asarray(mask, dtype=np.float64)
    return 0.5 * float(np.sum(np.abs(w) ** 2))


def born_hessian_norm(prob, iters=30, seed_vec=None):
    """Largest eigenvalue of sum_t Re{diag(u_in,t)^H H^H H diag(u_in,t)} by power iteration.

    This is the Lipschitz constant of the gradient of the first-Born
    (u = u_in) data term; the step size gamma = c / L is a reading (the paper
    tunes gamma by hand, Sec. IV).
    """
    shape = prob.u_in.shape[1:]
    x = np.ones(shape) if seed_vec is None else np.array(seed_vec, dtype=np.float64)
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = np.zeros(shape)
        for t in range(prob.T):
            Zt = prob.H @ (prob.u_in[t] * x).ravel()
            y += np.real(np.conj(prob.u_in[t]) * (np.conj(prob.H).T @ Zt).reshape(shape))
        lam = float(np.linalg.norm(y))
        x = y / lam
    return lam
