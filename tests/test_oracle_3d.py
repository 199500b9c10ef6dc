"""Pins of the oracle's 3D scalar model (Eq. 1 with d = 3): dense Toeplitz,
dense LU, the scalar Mie series of a sphere, the 3D TV prox closed form and
finite differences of the gradient."""
import math

import numpy as np
import pytest

from oracle import grad, mie, model, prox, solve
from paper_1708_01663_gb300 import synth

K, KB = model.wavenumbers(1.0)


def _dirs(T):
    th = np.linspace(0.3, 1.2, T)
    ph = np.linspace(0.0, 2.5, T)
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)


def test_fft_convolution_equals_dense_3d():
    n, delta = 4, 1.0 / 6
    G = model.green_matrix(n, delta, K, KB, dim=3)
    ghat = model.green_spectrum(n, 2 * n, delta, K, KB, dim=3)
    x = synth.random_field(3, (n, n, n))
    ref = (G @ x.ravel()).reshape(n, n, n)
    assert np.linalg.norm(model.conv_G(x, ghat, n) - ref) / np.linalg.norm(ref) < 1e-13
    refh = (G.conj().T @ x.ravel()).reshape(n, n, n)
    assert np.linalg.norm(model.conv_G(x, ghat, n, adjoint=True) - refh) / np.linalg.norm(refh) < 1e-13
    # padding independence
    ghat2 = model.green_spectrum(n, 2 * n + 3, delta, K, KB, dim=3)
    assert np.linalg.norm(model.conv_G(x, ghat2, n) - ref) / np.linalg.norm(ref) < 1e-13


def test_self_term_3d_matches_ball_integral():
    from scipy import integrate
    delta = 1.0 / 6
    a = delta * (3 / (4 * math.pi)) ** (1 / 3)
    re = integrate.quad(lambda r: (np.exp(1j * KB * r) / (4 * math.pi * r)).real * 4 * math.pi * r * r, 0, a)[0]
    im = integrate.quad(lambda r: (np.exp(1j * KB * r) / (4 * math.pi * r)).imag * 4 * math.pi * r * r, 0, a)[0]
    assert abs(model.self_term(K, KB, delta, dim=3) - K * K * (re + 1j * im)) < 1e-12


def test_solve_matches_dense_lu_3d():
    n, delta = 8, 1.0 / 6
    f = synth.sphere_phantom(n, 3, (0.2, 0.6), 4, 0.02)
    prob = model.Problem(n, delta, _dirs(2), np.array([[0.0, 0.0, 3.0]]), dim=3)
    A = np.eye(n ** 3) - model.green_matrix(n, delta, K, KB, dim=3) * f.ravel()[None, :]
    u, _, _ = solve.solve_fields(prob, f, prob.u_in, tol=1e-12)
    for t in range(2):
        ref = solve.solve_dense(A, prob.u_in[t].ravel())
        assert np.linalg.norm(u[t].ravel() - ref) / np.linalg.norm(ref) < 1e-10


def _mie3(n, delta, contrast=0.1, radius=1.0, sign=1.0):
    c = (np.arange(1, n + 1) - n / 2 - 0.5) * delta
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    f = np.where(X * X + Y * Y + Z * Z <= radius * radius, contrast, 0.0).astype(np.complex128)
    phi = np.linspace(0, 2 * np.pi, 12, endpoint=False)
    rx = np.stack([3.5 * np.cos(phi), 3.5 * np.sin(phi), 0.8 * np.cos(3 * phi)], axis=1)
    prob = model.Problem(n, delta, np.array([[0.0, 0.0, 1.0]]), rx, dim=3)
    u, _, res = solve.solve_fields(prob, sign * f, prob.u_in, tol=1e-11)
    ysc = prob.sense(sign * f, u)[0]
    ref = mie.mie_sphere(rx, radius, contrast, K)
    return np.linalg.norm(ysc - ref) / np.linalg.norm(ref)


def test_mie_sphere_and_refinement():
    # staircase voxels of a sphere: 15 % at lambda/6, 6 % at lambda/10
    e6 = _mie3(14, 1.0 / 6)
    e10 = _mie3(24, 1.0 / 10)
    assert e6 < 0.2
    assert e10 < 0.08
    assert e10 < 0.6 * e6
    # a planted sign error (f -> -f) is far off
    assert _mie3(24, 1.0 / 10, sign=-1.0) > 0.5


def test_tv3_plateau_closed_form():
    W, a, b, lam = 16, 0.2, 1.0, 0.4
    z = np.full((4, 5, W), a)
    z[:, :, W // 2:] = b
    x = prox.fgp3(z, lam, 4000, -10, 10)
    assert np.abs(x[:, :, : W // 2] - (a + 2 * lam / W)).max() < 1e-6
    assert np.abs(x[:, :, W // 2:] - (b - 2 * lam / W)).max() < 1e-6


def test_grad3_adjoint():
    x = synth.random_field(1, (5, 6, 7)).real
    p = [synth.random_field(2 + i, (5, 6, 7)).real for i in range(3)]
    d = prox.grad3(x)
    assert abs(sum(np.sum(d[i] * p[i]) for i in range(3)) - np.sum(x * prox.grad3_adj(*p))) < 1e-12


def test_gradient_3d_central_differences():
    n, delta = 6, 1.0 / 6
    rx = np.array([[0.0, 0.0, 2.5], [2.0, 0.5, 0.0], [-1.5, 1.5, 1.0], [0.3, -2.2, -1.0]])
    prob = model.Problem(n, delta, _dirs(2), rx, dim=3)
    f = synth.sphere_phantom(n, 2, (0.1, 0.4), 5, 0.02)
    ft = synth.sphere_phantom(n, 2, (0.2, 0.5), 6, 0.02)
    _, y, _, _ = grad.forward(prob, ft, tol=1e-13)
    D, g = grad.data_and_grad(prob, f, y, tol=1e-13)
    h = 1e-6
    for idx in [(1, 2, 3), (3, 3, 3), (5, 0, 4)]:
        for unit in (1.0, 1j):
            fp = f.copy(); fp[idx] += h * unit
            fm = f.copy(); fm[idx] -= h * unit
            fd = (grad.data_term(prob, fp, y, 1e-13) - grad.data_term(prob, fm, y, 1e-13)) / (2 * h)
            an = g[idx].real if unit == 1.0 else g[idx].imag
            assert abs(fd - an) <= 1e-6 * np.abs(g).max()
