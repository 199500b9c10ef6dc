"""Pins of the oracle's adjoint-state gradient (Prop. 1, Eq. 12)."""
import numpy as np
import pytest

from oracle import grad, model
from paper_1708_01663_gb300 import synth


def _small_problem(n=12, T=2, M=8, imag=0.03):
    delta = 1.0 / 8
    f = synth.ellipse_phantom(n, 3, (0.1, 0.6), 31, imag)
    prob = model.Problem(n, delta, synth.plane_wave_angles(T), synth.circle_receivers(M, 2.5))
    f_true = synth.ellipse_phantom(n, 2, (0.2, 0.7), 32, imag)
    _, y, _, _ = grad.forward(prob, f_true, tol=1e-13)
    return prob, f, y


def test_gradient_matches_central_differences():
    prob, f, y = _small_problem()
    D, g = grad.data_and_grad(prob, f, y, tol=1e-13)
    h = 1e-6
    for (iy, ix) in [(3, 4), (6, 6), (9, 2), (0, 11)]:
        for part, unit in [("re", 1.0), ("im", 1j)]:
            fp = f.copy(); fp[iy, ix] += h * unit
            fm = f.copy(); fm[iy, ix] -= h * unit
            fd = (grad.data_term(prob, fp, y, 1e-13) - grad.data_term(prob, fm, y, 1e-13)) / (2 * h)
            an = g[iy, ix].real if part == "re" else g[iy, ix].imag
            assert abs(fd - an) <= 1e-6 * np.abs(g).max(), (iy, ix, part, fd, an)


def test_taylor_remainder_is_second_order():
    prob, f, y = _small_problem()
    D0, g = grad.data_and_grad(prob, f, y, tol=1e-13)
    d = synth.random_field(77, f.shape)
    slope_lin = np.sum(g.real * d.real + g.imag * d.imag)
    hs = np.array([1e-2, 5e-3, 2.5e-3])
    rem = [abs(grad.data_term(prob, f + h * d, y, 1e-13) - D0 - h * slope_lin) for h in hs]
    rates = np.diff(np.log(rem)) / np.diff(np.log(hs))
    assert np.all(np.abs(rates - 2.0) < 0.2), rates


def test_gradient_at_zero_contrast():
    # f = 0: A = I, u = u_in, v = 0, so g = conj(u_in) * H^H w
    prob, _, y = _small_problem()
    f0 = np.zeros((prob.n, prob.n), dtype=np.complex128)
    D, g = grad.data_and_grad(prob, f0, y, tol=1e-13)
    w = -y
    ref = np.zeros_like(g)
    for t in range(prob.T):
        ref += np.conj(prob.u_in[t]) * (np.conj(prob.H).T @ w[t]).reshape(prob.n, prob.n)
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()
    assert abs(D - 0.5 * np.sum(np.abs(y) ** 2)) <= 1e-12 * D


def test_sensing_adjoint_identity():
    prob, f, _ = _small_problem()
    x = synth.random_field(3, (prob.n * prob.n,))
    w = synth.random_field(4, (prob.H.shape[0],))
    assert abs(np.vdot(w, prob.H @ x) - np.vdot(np.conj(prob.H).T @ w, x)) < 1e-12 * np.abs(prob.H).sum()
