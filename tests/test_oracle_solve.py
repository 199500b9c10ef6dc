"""Pins of the oracle's field solves (Eq. 13): dense LU, Born limit, reciprocity."""
import numpy as np
import pytest

from oracle import model, solve
from paper_1708_01663_gb300 import synth

K, KB = model.wavenumbers(1.0)


@pytest.mark.parametrize("n,contrast,imag", [(16, (0.0, 0.5), 0.0), (24, (0.0, 1.0), 0.05)])
def test_krylov_solve_matches_dense_lu(n, contrast, imag):
    delta = 1.0 / 8
    f = synth.ellipse_phantom(n, 4, contrast, 21, imag)
    prob = model.Problem(n, delta, synth.plane_wave_angles(3), synth.circle_receivers(8, 3.0))
    G = model.green_matrix(n, delta, K, KB)
    A = np.eye(n * n) - G * f.ravel()[None, :]
    u, its, res = solve.solve_fields(prob, f, prob.u_in, tol=1e-12)
    for t in range(3):
        ref = solve.solve_dense(A, prob.u_in[t].ravel())
        assert np.linalg.norm(u[t].ravel() - ref) / np.linalg.norm(ref) < 1e-10
    # adjoint system A^H v = b
    b = synth.random_field(4, (1, n, n))
    v, _, _ = solve.solve_fields(prob, f, b, tol=1e-12, adjoint=True)
    refv = solve.solve_dense(A.conj().T, b[0].ravel())
    assert np.linalg.norm(v[0].ravel() - refv) / np.linalg.norm(refv) < 1e-10


def test_gmres_matches_dense_lu():
    n, delta = 16, 1.0 / 8
    f = synth.ellipse_phantom(n, 3, (0.0, 0.8), 5)
    prob = model.Problem(n, delta, synth.plane_wave_angles(1), synth.circle_receivers(4, 3.0))
    A = np.eye(n * n) - model.green_matrix(n, delta, K, KB) * f.ravel()[None, :]
    apply = lambda v: prob.A(f, v.reshape(n, n)).ravel()
    x, _, res = solve.gmres(apply, prob.u_in[0].ravel(), tol=1e-12, restart=20)
    ref = solve.solve_dense(A, prob.u_in[0].ravel())
    assert res < 1e-11
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-10


def _born_gap(c):
    n, delta = 32, 1.0 / 8
    shape = synth.ellipse_phantom(n, 3, (1.0, 1.0), 9)
    f = c * shape
    prob = model.Problem(n, delta, synth.plane_wave_angles(2), synth.circle_receivers(4, 4.0))
    u, _, _ = solve.solve_fields(prob, f, prob.u_in, tol=1e-13)
    born = model.conv_G(f * prob.u_in, prob.ghat, n)
    return np.linalg.norm(u - prob.u_in - born) / np.linalg.norm(born)


def test_first_born_limit_is_linear_in_contrast():
    g1 = _born_gap(1e-4)
    g2 = _born_gap(0.5e-4)
    assert g1 < 1e-3
    assert abs(g1 / g2 - 2.0) < 0.2


def test_reciprocity_point_sources():
    n, delta = 24, 1.0 / 8
    f = synth.ellipse_phantom(n, 4, (0.0, 0.6), 13, imag=0.02)
    pos = np.array([[3.0, 0.5], [-1.0, 2.8], [0.4, -3.3]])
    u_in = model.point_sources(pos, n, delta, KB)
    prob = model.Problem(n, delta, None, pos, u_in=u_in)
    u, _, _ = solve.solve_fields(prob, f, u_in, tol=1e-13)
    Y = prob.sense(f, u)          # Y[t, r]: field at position r from a source at position t
    assert np.abs(Y - Y.T).max() / np.abs(Y).max() < 1e-9
