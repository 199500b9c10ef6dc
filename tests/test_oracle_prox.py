"""Pins of the oracle's constrained isotropic-TV prox (Eq. 8 through FGP)."""
import numpy as np
import pytest

from oracle import prox
from paper_1708_01663_gb300 import synth


def test_adjoint_of_difference_operator():
    x = synth.random_field(1, (9, 13)).real
    px = synth.random_field(2, (9, 13)).real
    py = synth.random_field(3, (9, 13)).real
    dx, dy = prox.grad2(x)
    assert abs(np.sum(dx * px + dy * py) - np.sum(x * prox.grad2_adj(px, py))) < 1e-12


def test_zero_weight_is_clamp():
    z = 2.0 * synth.random_field(5, (16, 16)).real
    assert np.array_equal(prox.fgp(z, 0.0, 20, 0.0, 2.0), np.clip(z, 0.0, 2.0))


def test_constant_image():
    z = np.full((12, 12), 2.7)
    assert np.allclose(prox.fgp(z, 0.3, 20, 0.0, 2.0), 2.0, atol=1e-15)
    z = np.full((12, 12), 0.7)
    assert np.allclose(prox.fgp(z, 0.3, 20, 0.0, 2.0), 0.7, atol=1e-15)


def test_two_plateau_closed_form():
    # Image constant along y, value a on the left W/2 columns and b on the right:
    # the prox reduces to 1D TV, where each plateau moves by lam / (its length).
    W, rows, a, b, lam = 16, 8, 0.2, 1.0, 0.4
    z = np.full((rows, W), a)
    z[:, W // 2:] = b
    x = prox.fgp(z, lam, 4000, -10.0, 10.0)
    assert np.abs(x[:, : W // 2] - (a + 2 * lam / W)).max() < 1e-6
    assert np.abs(x[:, W // 2:] - (b - 2 * lam / W)).max() < 1e-6


def test_two_plateau_rejects_doubled_weight():
    # a planted slip (TV weight 2 lam, i.e. a dropped 1/2 on the data term) misses the closed form
    W, rows, a, b, lam = 16, 8, 0.2, 1.0, 0.4
    z = np.full((rows, W), a)
    z[:, W // 2:] = b
    x2 = prox.fgp(z, 2 * lam, 4000, -10.0, 10.0)
    assert np.abs(x2[:, : W // 2] - (a + 2 * lam / W)).max() > 1e-2


def _objective(x, z, lam):
    return 0.5 * np.sum((x - z) ** 2) + lam * prox.tv_iso(x)


def test_local_optimality_and_box():
    z = synth.ellipse_phantom(20, 4, (0.0, 1.0), 3).real + 0.1 * synth.random_field(9, (20, 20)).real
    lam = 0.05
    x = prox.fgp(z, lam, 3000, 0.0, 0.9)
    assert x.min() >= 0.0 and x.max() <= 0.9
    base = _objective(x, z, lam)
    for s in range(20):
        d = 1e-3 * synth.random_field(100 + s, (20, 20)).real
        xp = np.clip(x + d, 0.0, 0.9)
        assert _objective(xp, z, lam) >= base - 1e-9


def test_non_expansive():
    z1 = synth.random_field(1, (16, 16)).real
    z2 = z1 + 0.3 * synth.random_field(2, (16, 16)).real
    x1 = prox.fgp(z1, 0.2, 2000, -0.5, 0.5)
    x2 = prox.fgp(z2, 0.2, 2000, -0.5, 0.5)
    assert np.linalg.norm(x1 - x2) <= np.linalg.norm(z1 - z2) + 1e-9


def test_objective_decreases_with_iterations():
    z = synth.ellipse_phantom(24, 4, (0.0, 1.0), 4).real + 0.2 * synth.random_field(3, (24, 24)).real
    lam = 0.1
    vals = [_objective(prox.fgp(z, lam, k, 0.0, 2.0), z, lam) for k in (5, 20, 100, 1000)]
    assert vals[-1] <= min(vals) + 1e-12
    assert vals[1] - vals[-1] < 0.1 * (vals[0] - vals[-1] + 1e-12) + 1e-3
