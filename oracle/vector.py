"""3D vectorial model of the appendix ("3D Diffractive Imaging") in FP64.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU
legs use this package.

Fields are E = (E^(1), E^(2), E^(3)), stored [3, n, n, n] per transmitter
(component, then z, y, x with x fastest).  With B^(c) = G~ (f E^(c)) the scalar
convolution of the appendix (G~_ij = delta^3 g(|r_i - r_j|), the 3D g of Eq. 1),
the discrete constraint and measurements are

    E = E_in + (k^2 I + D) B                       (appendix, discrete constraint)
    y = H~ (I_3 (x) diag f) E                      (appendix, discrete measurement)

D is the finite-difference grad-div operator printed in the appendix: the
3-point second difference for d^2/dx_c^2 and the 4-point diagonal stencil /
(4 delta^2) for the mixed derivatives.  H~ [M, 3N] holds the third row of the
dyadic Green's function (the receivers measure the z component), times delta^3.
Readings (the appendix is silent on them):
  * D acts on grid values only (it is a 3N x 3N matrix): neighbours outside
    the grid count as zero;
  * G~'s singular self term is the integral of g over the voxel's
    equal-volume ball, as in the scalar model (oracle.model.self_term / k^2);
  * eps_b = 1 (the appendix writes k^2 with the vacuum k);
  * incident fields are polarised plane waves p_t exp(j k d_t . r), p_t . d_t = 0.
With C = k^2 B = conv_G(f E) (G the scalar model's k^2-weighted matrix):
    A x   = x - C - D C / k^2
    A^H x = x - conj(f) conv_{G^H}(x + D x / k^2)     (D is real and symmetric)
Gradient (appendix, CISOR for 3D): with w = Z - y, z = H~^H w,
A^H v = conj(f) z, g = sum_c conj(E^(c)) (z^(c) + conv_{G^H}((I + D / k^2) v)^(c)),
grad D = Re g for real f.

Pinned by: a dense 3N x 3N matrix built from the printed stencils and the
dense scalar G (tests/test_oracle_vector.py), central differences of D, and
the Clausius-Mossotti dipole of a small dielectric sphere (a planted missing
grad-div term fails it).
"""
from __future__ import annotations

import math

import numpy as np

from . import model
from .solve import bicgstab


def dyadic_third_row(rx: np.ndarray, n: int, delta: float, k: float) -> np.ndarray:
    """H~ [M, 3N]: delta^3 times row 3 of the dyadic Green's function
    G(r) = k^2 [ (3/(k d)^2 - 3j/(k d) - 1) r^ r^T + (1 + j/(k d) - 1/(k d)^2) I ] g(d)."""
    pts = model.grid_points(n, delta, 3)
    dv = np.asarray(rx, dtype=np.float64)[:, None, :] - pts[None, :, :]
    d = np.sqrt((dv ** 2).sum(-1))
    rh = dv / d[..., None]
    g = np.exp(1j * k * d) / (4.0 * math.pi * d)
    kd = k * d
    a = 3.0 / kd ** 2 - 3j / kd - 1.0
    b = 1.0 + 1j / kd - 1.0 / kd ** 2
    out = np.empty((len(rx), 3, pts.shape[0]), dtype=np.complex128)
    for c in range(3):
        out[:, c, :] = k * k * (a * rh[..., 2] * rh[..., c] + (b if c == 2 else 0.0)) * g
    return delta ** 3 * out.reshape(len(rx), 3 * pts.shape[0])


def polarised_plane_waves(dirs: np.ndarray, pols: np.ndarray, n: int, delta: float, k: float) -> np.ndarray:
    """[T, 3, n, n, n] incident fields p_t exp(j k d_t . r)."""
    scal = model.plane_waves_3d(dirs, n, delta, k)
    return np.asarray(pols, dtype=np.float64)[:, :, None, None, None] * scal[:, None]


def graddiv(B: np.ndarray, delta: float) -> np.ndarray:
    """(D B)^(c) = sum_j d_c d_j B^(j) with the appendix's stencils, zero outside the grid.
    B: [3, n, n, n] with axes (z, y, x); component c differentiates along x (c = 0), y, z."""
    n = B.shape[1]
    P = np.zeros((3, n + 2, n + 2, n + 2), dtype=np.complex128)
    P[:, 1:-1, 1:-1, 1:-1] = B
    ax = {0: 3, 1: 2, 2: 1}  # component -> array axis of P (x is the last)

    def sh(a, offs):
        """a shifted so that out[p] = a[p + offs] on the interior (offs per component direction)."""
        sl = [slice(1, -1)] * 3
        for comp, o in offs.items():
            axis = ax[comp] - 1
            sl[axis] = slice(1 + o, n + 1 + o)
        return a[tuple(sl)]

    out = np.zeros_like(B, dtype=np.complex128)
    for c in range(3):
        acc = (sh(P[c], {c: 1}) - 2.0 * sh(P[c], {}) + sh(P[c], {c: -1})) / delta ** 2
        for j in range(3):
            if j == c:
                continue
            acc = acc + (sh(P[j], {c: -1, j: -1}) - sh(P[j], {c: -1, j: 1}) - sh(P[j], {c: 1, j: -1})
                         + sh(P[j], {c: 1, j: 1})) / (4.0 * delta ** 2)
        out[c] = acc
    return out


class VectorProblem:
    """Tables of one vectorial geometry: ghat (scalar 3D spectrum, k^2-weighted), H~, E_in."""

    def __init__(self, n: int, delta: float, dirs, pols, rx, wavelength: float = 1.0, P: int | None = None):
        self.n, self.delta = n, delta
        self.k, _ = model.wavenumbers(wavelength, 1.0)
        self.P = P if P is not None else 2 * n
        self.ghat = model.green_spectrum(n, self.P, delta, self.k, self.k, 3)
        self.rx = np.asarray(rx, dtype=np.float64)
        self.H = dyadic_third_row(self.rx, n, delta, self.k)
        self.u_in = polarised_plane_waves(np.asarray(dirs), np.asarray(pols), n, delta, self.k)
        self.T = self.u_in.shape[0]

    def conv(self, x, adjoint=False):
        return np.stack([model.conv_G(x[c], self.ghat, self.n, adjoint=adjoint) for c in range(3)])

    def A(self, f, x):
        C = self.conv(f[None] * x)
        return x - C - graddiv(C, self.delta) / self.k ** 2

    def AH(self, f, x):
        w = x + graddiv(x, self.delta) / self.k ** 2
        return x - np.conj(f)[None] * self.conv(w, adjoint=True)

    def sense(self, f, E):
        """Z[t, m] = H~ (I_3 (x) diag f) E_t."""
        return np.stack([self.H @ (f[None] * E[t]).ravel() for t in range(E.shape[0])])


def solve_fields(prob, f, B, tol=1e-10, adjoint=False, x0=None):
    shape = (3,) + f.shape
    op = prob.AH if adjoint else prob.A
    apply = lambda v: op(f, v.reshape(shape)).ravel()
    out = np.empty(B.shape, dtype=np.complex128)
    for t in range(B.shape[0]):
        g = None if x0 is None else x0[t].ravel()
        x, _, _ = bicgstab(apply, B[t].ravel(), g, tol, 20000)
        out[t] = x.reshape(shape)
    return out


def data_and_grad(prob, f, y, tol=1e-10):
    """D(f) = 1/2 sum_t ||Z_t - y_t||^2 and g of the appendix's gradient (grad D = Re g for real f)."""
    u = solve_fields(prob, f, prob.u_in, tol)
    w = prob.sense(f, u) - y
    D = 0.5 * float(np.sum(np.abs(w) ** 2))
    g = np.zeros(f.shape, dtype=np.complex128)
    shape = (3,) + f.shape
    for t in range(prob.T):
        z = (np.conj(prob.H).T @ w[t]).reshape(shape)
        v = solve_fields(prob, f, (np.conj(f)[None] * z)[None], tol, adjoint=True)[0]
        gz = z + prob.conv(v + graddiv(v, prob.delta) / prob.k ** 2, adjoint=True)
        g += np.sum(np.conj(u[t]) * gz, axis=0)
    return D, g


def data_term(prob, f, y, tol=1e-12):
    u = solve_fields(prob, f, prob.u_in, tol)
    return 0.5 * float(np.sum(np.abs(prob.sense(f, u) - y) ** 2))
