"""Per-transmitter oracle work in a process pool, for the full-size parity tests.

D and Prop. 1's g are sums over transmitters and every transmitter's solves
are independent (Eq. 13), so the oracle runs one single-transmitter problem
per worker and the test sums the results (the identity the transmitter-split
tests pin).  The pool uses the spawn start method, which is safe after the
test process has initialised CUDA.  Imports only the oracle and the seeded
input generators.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from oracle import grad, model, solve


def pool(n):
    return mp.get_context("spawn").Pool(max(1, min(n, os.cpu_count() or 1)))


def _problem(geom, t):
    n, delta, angles, rx, P = geom
    return model.Problem(n, delta, np.asarray(angles)[[t]], rx, P=P)


def solve_one(args):
    """Field of transmitter t at contrast f (BiCGSTAB to tol) and its measurements H diag(u) f."""
    geom, t, f, tol = args
    prob = _problem(geom, t)
    u, its, res = solve.solve_fields(prob, f, prob.u_in, tol=tol)
    return u[0], prob.sense(f, u)[0], float(res[0])


def data_grad_one(args):
    """D_t and g_t (Prop. 1) of transmitter t at s, warm-started from u0, v0; also returns u_t, v_t."""
    geom, t, s, y_t, u0, v0, tol = args
    prob = _problem(geom, t)
    D, g, u, v = grad.data_and_grad(prob, s, y_t[None], tol=tol, u0=None if u0 is None else u0[None],
                                    v0=None if v0 is None else v0[None], return_fields=True)
    return D, g, u[0], v[0]
