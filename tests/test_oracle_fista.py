"""Pins of the oracle's relaxed FISTA (Eqs. 9-11)."""
import math

import numpy as np

from oracle import fista, grad, model, prox
from paper_1708_01663_gb300 import synth


def _born_model(n=6, T=4, M=16, radius=2.0):
    delta = 1.0 / 8
    prob = model.Problem(n, delta, synth.plane_wave_angles(T), synth.circle_receivers(M, radius))
    J = [prob.H * prob.u_in[t].ravel()[None, :] for t in range(T)]   # Z_t = H diag(u_in,t) f
    return prob, J


def test_alpha_zero_is_ista():
    prob, J = _born_model()
    n = prob.n
    f_true = synth.ellipse_phantom(n, 2, (0.3, 0.6), 2).real
    y = np.stack([Jt @ f_true.ravel() for Jt in J])

    def gfn(s, state):
        w = [Jt @ s.ravel() - y[t] for t, Jt in enumerate(J)]
        g = sum(np.conj(Jt).T @ w[t] for t, Jt in enumerate(J)).reshape(n, n)
        return 0.5 * sum(np.sum(np.abs(wt) ** 2) for wt in w), g

    L = grad.born_hessian_norm(prob)
    gamma, tau = 0.5 / L, 1e-3
    out, _ = fista.relaxed_fista(prob, y, np.zeros((n, n)), gamma, tau, 0.0, 15, 30, grad_fn=gfn)
    x = np.zeros((n, n))
    for _ in range(15):               # plain ISTA: x <- prox(x - gamma grad)
        _, g = gfn(x, None)
        x = prox.fgp(x - gamma * g.real, gamma * tau, 30, 0.0, 2.0)
    assert np.abs(out.real - x).max() < 1e-14


def test_linear_model_converges_to_least_squares():
    prob, J = _born_model(n=3, T=8, M=32, radius=0.5)
    n = prob.n
    rng_f = synth.random_field(5, (n, n)).real
    y = np.stack([Jt @ rng_f.ravel() for Jt in J]) + 0.01 * synth.complex_noise(6, (len(J), J[0].shape[0]))

    def gfn(s, state):
        w = [Jt @ s.real.ravel() - y[t] for t, Jt in enumerate(J)]
        g = sum(np.conj(Jt).T @ w[t] for t, Jt in enumerate(J)).reshape(n, n)
        return 0.5 * sum(np.sum(np.abs(wt) ** 2) for wt in w), g

    Jall = np.concatenate(J)
    Areal = np.concatenate([Jall.real, Jall.imag])
    breal = np.concatenate([y.ravel().real, y.ravel().imag])
    ls = np.linalg.lstsq(Areal, breal, rcond=None)[0].reshape(n, n)
    L = grad.born_hessian_norm(prob, iters=200)
    out, hist = fista.relaxed_fista(prob, y, np.zeros((n, n)), 1.0 / L, 0.0, 0.96, 2000, 1,
                                    box_re=(-np.inf, np.inf), grad_fn=gfn)
    assert np.linalg.norm(out.real - ls) / np.linalg.norm(ls) < 1e-8


def test_iterates_stay_in_box_and_objective_falls():
    prob, J = _born_model(n=8)
    n = prob.n
    f_true = synth.ellipse_phantom(n, 2, (0.5, 1.5), 8).real
    y = np.stack([Jt @ f_true.ravel() for Jt in J])

    def gfn(s, state):
        w = [Jt @ s.real.ravel() - y[t] for t, Jt in enumerate(J)]
        g = sum(np.conj(Jt).T @ w[t] for t, Jt in enumerate(J)).reshape(n, n)
        return 0.5 * sum(np.sum(np.abs(wt) ** 2) for wt in w), g

    L = grad.born_hessian_norm(prob)
    out, hist = fista.relaxed_fista(prob, y, np.zeros((n, n)), (1 - 0.96 ** 2) / (2 * L), 1e-3,
                                    0.96, 200, 20, box_re=(0.0, 1.0), grad_fn=gfn)
    assert out.real.min() >= 0.0 and out.real.max() <= 1.0
    assert hist[-1] < 0.5 * hist[0]


def test_nonlinear_reconstruction_improves_snr():
    # small noise-free nonlinear problem: CISOR raises the reconstructed SNR
    n, delta = 16, 1.0 / 8
    prob = model.Problem(n, delta, synth.plane_wave_angles(6), synth.circle_receivers(24, 3.0))
    f_true = synth.ellipse_phantom(n, 2, (0.05, 0.1), 41)
    _, y, _, _ = grad.forward(prob, f_true, tol=1e-12)
    L = grad.born_hessian_norm(prob)
    out, hist = fista.relaxed_fista(prob, y, np.zeros((n, n)), 1.0 / L, 1e-6, 0.96, 40, 10, tol=1e-9)
    assert hist[-1] < 0.05 * hist[0]
    assert fista.recon_snr_db(out, f_true) > 3.0
