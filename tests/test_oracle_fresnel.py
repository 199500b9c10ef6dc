"""Pins of the oracle's Fresnel-style geometry (Sec. IV): point-source
transmitters and per-transmitter receiver masks.

A masked data term must equal the sum, over transmitters, of sub-problems that
hold only that transmitter and its active receivers (H rebuilt from the kept
receiver positions: an independent construction of the masked operator).
Point sources: reciprocity Y[t, r] = Y[r, t] in 3D (2D in test_oracle_solve),
and the incident field's outgoing far-field phase."""
import numpy as np

from oracle import grad, model, solve
from paper_1708_01663_gb300 import synth

K, KB = model.wavenumbers(1.0)


def _fresnel_like(n=20, T=4, M=12, seed=3):
    delta = 1.0 / 8
    ang = 2 * np.pi * np.arange(T) / T
    src = np.stack([3.5 * np.cos(ang), 3.5 * np.sin(ang)], 1)
    phi = 2 * np.pi * np.arange(M) / M
    rx = np.stack([4.0 * np.cos(phi), 4.0 * np.sin(phi)], 1)
    # receivers more than 60 degrees from the source direction are active
    dang = np.abs((phi[None, :] - ang[:, None] + np.pi) % (2 * np.pi) - np.pi)
    mask = (dang > np.pi / 3).astype(np.float64)
    f = synth.ellipse_phantom(n, 3, (0.1, 0.6), seed, 0.03)
    return n, delta, src, rx, mask, f


def test_masked_gradient_equals_sum_of_receiver_subproblems():
    n, delta, src, rx, mask, f = _fresnel_like()
    prob = model.Problem(n, delta, src, rx, tx_kind="point")
    f_true = synth.ellipse_phantom(n, 3, (0.1, 0.7), 9, 0.03)
    _, y, _, _ = grad.forward(prob, f_true, tol=1e-12)
    D, g = grad.data_and_grad(prob, f, y, tol=1e-12, mask=mask)
    D_sum, g_sum = 0.0, np.zeros_like(g)
    for t in range(len(src)):
        keep = mask[t] > 0
        sub = model.Problem(n, delta, src[t:t + 1], rx[keep], tx_kind="point")
        Dt, gt = grad.data_and_grad(sub, f, y[t:t + 1, keep], tol=1e-12)
        D_sum += Dt
        g_sum += gt
    assert abs(D - D_sum) <= 1e-10 * D
    assert np.linalg.norm(g - g_sum) <= 1e-9 * np.linalg.norm(g)
    # the mask matters: the unmasked term differs
    D_all, _ = grad.data_and_grad(prob, f, y, tol=1e-12)
    assert D_all > (1 + 1e-3) * D
    assert abs(grad.data_term(prob, f, y, 1e-12, mask=mask) - D) <= 1e-9 * D


def test_point_sources_reciprocity_3d():
    n, delta = 8, 1.0 / 6
    f = synth.sphere_phantom(n, 2, (0.2, 0.5), 4, 0.02)
    pos = np.array([[2.5, 0.3, 0.2], [-0.4, 2.2, 0.9], [0.5, -0.7, -2.4]])
    prob = model.Problem(n, delta, pos, pos, tx_kind="point", dim=3)
    u, _, _ = solve.solve_fields(prob, f, prob.u_in, tol=1e-13)
    Y = prob.sense(f, u)
    assert np.abs(Y - Y.T).max() / np.abs(Y).max() < 1e-9


def test_point_source_field_is_outgoing():
    # far from a 2D line source, u_in ~ sqrt(2/(pi k r)) e^{j(k r + pi/4)} / (4j) ... phase advances by k dr
    src = np.array([[40.0, 0.0]])
    u = model.point_sources(src, 8, 1.0 / 8, KB)[0]
    # along x the distance to the source decreases, so the phase falls by k * delta per pixel
    dphi = np.angle(u[4, 1:] / u[4, :-1])
    assert np.allclose(dphi, -KB / 8, atol=2e-3)
