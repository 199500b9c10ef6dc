"""Relaxed FISTA (Sec. III-A, Eqs. 9-11).

    f_k     = prox_{gamma R}(s_k - gamma grad D(s_k))            (Eq. 9)
    t_{k+1} = (sqrt(4 t_k^2 + 1) + 1) / 2                        (Eq. 10)
    s_{k+1} = f_k + alpha ((t_k - 1) / t_{k+1}) (f_k - f_{k-1})  (Eq. 11)

The paper initialises "s_1 = f_0, t_0 = 1" while the recursion reads t_k from
k = 1; the reading taken is t_1 = 1 and s_1 = f_0.  alpha = 0 is ISTA and
alpha = 1 FISTA (Sec. III-A).  Inner solves start from the previous outer
iterate's fields (u_in and 0 on the first iteration).

Pinned by: alpha = 0 against a separately written ISTA loop, convergence to
the dense least-squares solution on a linear (first-Born) model, iterates in C
(tests/test_oracle_fista.py).  The full nonconvex trajectory has no
closed form: parity unpinned beyond these.
"""
from __future__ import annotations

import math

import numpy as np

from .grad import data_and_grad
from .prox import prox_R


def relaxed_fista(prob, y, f0, gamma, tau, alpha, iters, tv_iters, box_re=(0.0, 2.0),
                  box_im=None, tol=1e-10, grad_fn=None):
    """Run ``iters`` relaxed-FISTA steps from f0; returns f_K and the per-step D values.

    ``grad_fn(s, state) -> (D, g)`` replaces the nonlinear gradient (tests use
    it for linear models); g is Prop. 1's complex vector, whose real part is
    the gradient for real f and whose real/imaginary parts are the partial
    derivatives for complex f.
    """
    f_prev = np.array(f0, dtype=np.complex128)
    s = f_prev.copy()
    t = 1.0
    lam = gamma * tau
    hist = []
    state = {"u": None, "v": None}
    for _ in range(iters):
        if grad_fn is None:
            D, g, u, v = data_and_grad(prob, s, y, tol=tol, u0=state["u"], v0=state["v"],
                                       return_fields=True)
            state["u"], state["v"] = u, v
        else:
            D, g = grad_fn(s, state)
        step = g.real if box_im is None else g
        f = prox_R(s - gamma * step, lam, tv_iters, box_re, box_im)
        t_new = (math.sqrt(4.0 * t * t + 1.0) + 1.0) / 2.0
        s = f + alpha * ((t - 1.0) / t_new) * (f - f_prev)
        f_prev, t = f, t_new
        hist.append(D)
    return f_prev, hist


def recon_snr_db(f_hat, f_true):
    """Reconstructed SNR 20 log10(||f_true|| / ||f_hat - f_true||) (Sec. IV)."""
    return 20.0 * math.log10(np.linalg.norm(f_true) / np.linalg.norm(f_hat - f_true))
