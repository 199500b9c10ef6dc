"""Pins of the oracle's discretised model (Sec. II, Eqs. 1-5) against things other than itself."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import mie, model, solve
from paper_1708_01663_gb300 import synth

K, KB = model.wavenumbers(1.0)


def _dense_G_by_loops(n, delta):
    """G by an explicit double loop over pixel pairs (the Toeplitz definition)."""
    c = (np.arange(1, n + 1) - n / 2.0 - 0.5) * delta
    pts = [(c[ix], c[iy]) for iy in range(n) for ix in range(n)]
    N = len(pts)
    G = np.zeros((N, N), dtype=np.complex128)
    for i in range(N):
        for j in range(N):
            if i == j:
                G[i, j] = model.self_term(K, KB, delta)
            else:
                r = math.hypot(pts[i][0] - pts[j][0], pts[i][1] - pts[j][1])
                G[i, j] = K * K * delta * delta * 0.25j * complex(special.hankel1(0, KB * r))
    return G


@pytest.mark.parametrize("n", [5, 8])
def test_fft_convolution_equals_dense_toeplitz(n):
    delta = 1.0 / 8
    G = _dense_G_by_loops(n, delta)
    ghat = model.green_spectrum(n, 2 * n, delta, K, KB)
    x = synth.random_field(11, (n, n))
    ref = (G @ x.ravel()).reshape(n, n)
    got = model.conv_G(x, ghat, n)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13
    # G^H through conj(ghat)
    refh = (G.conj().T @ x.ravel()).reshape(n, n)
    goth = model.conv_G(x, ghat, n, adjoint=True)
    assert np.linalg.norm(goth - refh) / np.linalg.norm(refh) < 1e-13


def test_dense_G_is_symmetric_not_hermitian():
    G = model.green_matrix(6, 1.0 / 8, K, KB)
    assert np.abs(G - G.T).max() < 1e-14
    assert np.abs(G - G.conj().T).max() > 1e-3


@pytest.mark.parametrize("P_extra", [1, 6, 11])
def test_padding_independence(P_extra):
    n, delta = 12, 1.0 / 8
    x = synth.random_field(5, (n, n))
    a = model.conv_G(x, model.green_spectrum(n, 2 * n, delta, K, KB), n)
    b = model.conv_G(x, model.green_spectrum(n, 2 * n + P_extra, delta, K, KB), n)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-13


def test_adjoint_identity_of_A():
    n, delta = 16, 1.0 / 8
    ghat = model.green_spectrum(n, 2 * n, delta, K, KB)
    f = synth.ellipse_phantom(n, 3, (0.0, 0.5), 3, imag=0.05)
    x = synth.random_field(1, (n, n))
    y = synth.random_field(2, (n, n))
    lhs = np.vdot(y, model.apply_A(f, x, ghat))
    rhs = np.vdot(model.apply_AH(f, y, ghat), x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13


def test_self_term_matches_quadrature():
    # closed form of the disk integral vs adaptive quadrature of g over the disk
    delta = 1.0 / 8
    a = delta / math.sqrt(math.pi)
    re = integrate.quad(lambda r: (0.25j * special.hankel1(0, KB * r)).real * 2 * math.pi * r, 0, a, limit=200)[0]
    im = integrate.quad(lambda r: (0.25j * special.hankel1(0, KB * r)).imag * 2 * math.pi * r, 0, a,
                        points=[0.0], limit=200)[0]
    ref = K * K * (re + 1j * im)
    assert abs(model.self_term(K, KB, delta) - ref) / abs(ref) < 1e-8


def test_green_far_field_is_outgoing():
    # (j/4) H0^(1)(kr) ~ (j/4) sqrt(2/(pi k r)) e^{j(kr - pi/4)} for kr >> 1
    r = 200.0
    asym = 0.25j * math.sqrt(2.0 / (math.pi * KB * r)) * np.exp(1j * (KB * r - math.pi / 4))
    assert abs(model.green(r, KB) - asym) / abs(asym) < 1e-3


def _mie_error(n, delta, contrast, radius=1.0, sign=1.0):
    f = synth.disk_phantom(n, delta, radius, contrast)
    rx = synth.circle_receivers(32, 3.0)
    prob = model.Problem(n, delta, np.array([0.0]), rx)
    u, _, res = solve.solve_fields(prob, sign * f, prob.u_in, tol=1e-12)
    assert res.max() < 1e-10
    ysc = prob.sense(sign * f, u)[0]
    ref = mie.mie_cylinder(rx, radius, contrast, K)
    return np.linalg.norm(ysc - ref) / np.linalg.norm(ref)


def test_mie_cylinder_and_refinement():
    e8 = _mie_error(24, 1 / 8, 0.1)
    e16 = _mie_error(48, 1 / 16, 0.1)
    e32 = _mie_error(96, 1 / 32, 0.1)
    assert e8 < 0.05
    assert e16 < e8 and e32 < e16
    assert e32 < 0.01


def test_mie_higher_contrast():
    assert _mie_error(64, 1 / 16, 0.5) < 0.05


def test_mie_rejects_opposite_green_sign():
    # -(j/4) H0 is the same as f -> -f: a planted sign error must fail the pin
    assert _mie_error(48, 1 / 16, 0.1, sign=-1.0) > 0.5
