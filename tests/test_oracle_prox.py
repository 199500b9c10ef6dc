"""Pins of the oracle's constrained isotropic-TV prox (Eq. 8 through FGP)."""
import math

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


# ---------------------------------------------------------------- anisotropic TV (parallel proximal)
def _aniso_dual_reference(z, lam, iters=20000):
    """Exact prox of lam * TV_aniso (no box) by accelerated projected gradient on
    the dual: x = z - D^T p, p_d in [-lam, lam] per pixel (a different algorithm)."""
    nd = z.ndim
    def D(x):
        out = []
        for a in range(nd):
            d = np.zeros_like(x)
            sl_hi = [slice(None)] * nd; sl_hi[a] = slice(1, None)
            sl_lo = [slice(None)] * nd; sl_lo[a] = slice(None, -1)
            d[tuple(sl_lo)] = x[tuple(sl_hi)] - x[tuple(sl_lo)]
            out.append(d)
        return out
    def DT(ps):
        out = np.zeros_like(ps[0])
        for a, p in enumerate(ps):
            sl_hi = [slice(None)] * nd; sl_hi[a] = slice(1, None)
            sl_lo = [slice(None)] * nd; sl_lo[a] = slice(None, -1)
            out[tuple(sl_lo)] -= p[tuple(sl_lo)]
            out[tuple(sl_hi)] += p[tuple(sl_lo)]
        return out
    p = [np.zeros_like(z) for _ in range(nd)]
    q = [pi.copy() for pi in p]
    t = 1.0
    step = 1.0 / (4.0 * nd)
    for _ in range(iters):
        g = D(z - DT(q))
        pn = [np.clip(qi + step * gi, -lam, lam) for qi, gi in zip(q, g)]
        tn = (1 + math.sqrt(1 + 4 * t * t)) / 2
        q = [a + ((t - 1) / tn) * (a - b) for a, b in zip(pn, p)]
        p, t = pn, tn
    return z - DT(p)


@pytest.mark.parametrize("shape", [(12, 10), (6, 5, 7)])
def test_ppa_aniso_converges_to_exact_prox(shape):
    z = synth.random_field(31, shape).real
    lam = 0.3
    ref = _aniso_dual_reference(z, lam)
    x = prox.ppa_aniso(z, lam, 3000)
    assert np.abs(x - ref).max() < 1e-5
    # optimality margin: the reference is the minimiser of the prox objective
    obj = lambda v: 0.5 * np.sum((v - z) ** 2) + lam * prox.tv_aniso(v)
    assert abs(obj(x) - obj(ref)) < 1e-8 * obj(ref) + 1e-10


def test_ppa_aniso_wrong_threshold_fails():
    # a planted mistake (threshold lam instead of m lam in the pieces) does not reach the prox
    z = synth.random_field(32, (10, 9)).real
    ref = _aniso_dual_reference(z, 0.3)
    pieces = [(a, par) for a in range(2) for par in (0, 1)]
    zs = [z.copy() for _ in range(5)]
    for _ in range(2000):
        ps = [prox.pair_shrink(zs[j], a, par, 0.3) for j, (a, par) in enumerate(pieces)] + [zs[-1]]
        x = sum(ps) / 5
        zs = [x + zj - pj for zj, pj in zip(zs, ps)]
    assert np.abs(x - ref).max() > 1e-2


def test_ppa_aniso_plateau_closed_form_and_limits():
    W, a, b, lam = 16, 0.2, 1.0, 0.4
    z = np.full((5, W), a)
    z[:, W // 2:] = b
    x = prox.ppa_aniso(z, lam, 4000, -10, 10)
    assert np.abs(x[:, : W // 2] - (a + 2 * lam / W)).max() < 1e-6
    assert np.abs(x[:, W // 2:] - (b - 2 * lam / W)).max() < 1e-6
    zz = synth.random_field(5, (8, 8)).real
    assert np.array_equal(prox.ppa_aniso(zz, 0.0, 10, -0.5, 0.5), np.clip(zz, -0.5, 0.5))
    c = np.full((6, 7), 0.7)
    assert np.allclose(prox.ppa_aniso(c, 0.5, 50, 0.0, 2.0), c, atol=1e-12)


def test_ppa_aniso_respects_box():
    z = 2.0 * synth.random_field(33, (9, 9)).real
    x = prox.ppa_aniso(z, 0.1, 3000, -0.5, 0.8)
    # Dykstra-type iterations reach the box only in the limit
    assert x.min() > -0.5 - 1e-4 and x.max() < 0.8 + 1e-4
