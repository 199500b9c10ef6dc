"""Pins of the oracle's 3D vectorial model (appendix, "3D Diffractive Imaging").

* The FFT/stencil operator equals the dense 3N x 3N matrix
  I - (k^2 I + D)(I_3 (x) G~ diag f), with D assembled by loops from the printed
  finite-difference stencils and G~ from the dense scalar Green's matrix.
* Central differences of D(f) against the appendix's gradient.
* Physics: a small dielectric sphere scatters as a dipole with the
  Clausius-Mossotti moment p = V f 3/(eps + 2) E_in (V the voxelised volume);
  dropping the grad-div term (a planted mistake) gives p = V f E_in instead and
  fails by (eps + 2)/3.
"""
import math

import numpy as np
import pytest

from oracle import model, vector
from paper_1708_01663_gb300 import synth

K, _ = model.wavenumbers(1.0)


def _dense_graddiv(n, delta):
    N = n ** 3
    D = np.zeros((3 * N, 3 * N))
    idx = lambda x, y, z: (z * n + y) * n + x
    for z in range(n):
        for y in range(n):
            for x in range(n):
                p = [x, y, z]
                for c in range(3):
                    row = c * N + idx(x, y, z)
                    for s, w in ((1, 1.0), (0, -2.0), (-1, 1.0)):
                        q = list(p)
                        q[c] += s
                        if all(0 <= v < n for v in q):
                            D[row, c * N + idx(*q)] += w / delta ** 2
                    for j in range(3):
                        if j == c:
                            continue
                        for sc, sj, w in ((-1, -1, 1.0), (-1, 1, -1.0), (1, -1, -1.0), (1, 1, 1.0)):
                            q = list(p)
                            q[c] += sc
                            q[j] += sj
                            if all(0 <= v < n for v in q):
                                D[row, j * N + idx(*q)] += w / (4.0 * delta ** 2)
    return D


def test_operator_equals_dense_matrix():
    n, delta = 4, 1.0 / 6
    rng_dirs = np.array([[0.0, 0.0, 1.0]])
    prob = vector.VectorProblem(n, delta, rng_dirs, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 0.0, 2.0]]))
    f = synth.sphere_phantom(n, 2, (0.2, 0.7), 3, 0.05)
    Gt = model.green_matrix(n, delta, K, K, dim=3) / K ** 2
    D = _dense_graddiv(n, delta)
    N = n ** 3
    blk = Gt * f.ravel()[None, :]
    A = np.eye(3 * N) - (K ** 2 * np.eye(3 * N) + D) @ np.kron(np.eye(3), blk)
    x = synth.random_field(7, (3, n, n, n))
    ref = (A @ x.ravel()).reshape(3, n, n, n)
    assert np.linalg.norm(prob.A(f, x) - ref) / np.linalg.norm(ref) < 1e-12
    refh = (A.conj().T @ x.ravel()).reshape(3, n, n, n)
    assert np.linalg.norm(prob.AH(f, x) - refh) / np.linalg.norm(refh) < 1e-12
    # D is real and symmetric (so D^H = D in A^H)
    assert np.abs(D - D.T).max() == 0.0


def test_gradient_central_differences():
    n, delta = 5, 1.0 / 6
    dirs = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]])
    pols = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    rx = np.array([[0.2, 0.1, 2.5], [2.2, -0.4, 0.3], [-1.8, 1.1, 0.9], [0.5, -2.1, -1.0]])
    prob = vector.VectorProblem(n, delta, dirs, pols, rx)
    f = synth.sphere_phantom(n, 2, (0.1, 0.4), 5, 0.02)
    ft = synth.sphere_phantom(n, 2, (0.2, 0.5), 6, 0.02)
    u = vector.solve_fields(prob, ft, prob.u_in, tol=1e-13)
    y = prob.sense(ft, u)
    D, g = vector.data_and_grad(prob, f, y, tol=1e-13)
    h = 1e-6
    for idx in [(1, 2, 3), (2, 2, 2), (4, 0, 1)]:
        for unit in (1.0, 1j):
            fp = f.copy(); fp[idx] += h * unit
            fm = f.copy(); fm[idx] -= h * unit
            fd = (vector.data_term(prob, fp, y, 1e-13) - vector.data_term(prob, fm, y, 1e-13)) / (2 * h)
            an = g[idx].real if unit == 1.0 else g[idx].imag
            assert abs(fd - an) <= 1e-6 * np.abs(g).max()


def _sphere_dipole(drop_graddiv=False):
    eps = 3.0
    a, delta = 0.03, 0.005
    n = 14
    c = (np.arange(n) - n / 2 + 0.5) * delta
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    f = np.where(X ** 2 + Y ** 2 + Z ** 2 <= a * a, eps - 1.0, 0.0).astype(np.complex128)
    V = np.count_nonzero(f) * delta ** 3
    phi = np.linspace(0, 2 * np.pi, 8, endpoint=False)
    rx = np.stack([2.0 * np.cos(phi), 2.0 * np.sin(phi), 0.7 * np.sin(2 * phi)], 1)
    prob = vector.VectorProblem(n, delta, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 0.0, 1.0]]), rx)
    if drop_graddiv:
        prob.A = lambda ff, x: x - prob.conv(ff[None] * x)
    E = vector.solve_fields(prob, f, prob.u_in, tol=1e-11)
    y = prob.sense(f, E)[0]
    # dipole at the origin: E_z(r) = (row 3 of the dyadic G)(r) p / delta^3 per unit delta^3 weight
    p = V * (eps - 1.0) * 3.0 / (eps + 2.0) * np.array([0.0, 0.0, 1.0])
    Hd = vector.dyadic_third_row(rx, 1, 1.0, K)  # one "voxel" of unit volume at the origin
    ref = Hd.reshape(len(rx), 3) @ p
    return np.linalg.norm(y - ref) / np.linalg.norm(ref)


def test_small_sphere_is_a_clausius_mossotti_dipole():
    err = _sphere_dipole()
    assert err < 0.08, err
    assert _sphere_dipole(drop_graddiv=True) > 0.4
