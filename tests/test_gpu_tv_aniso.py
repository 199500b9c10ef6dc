"""Anisotropic TV prox (parallel proximal algorithm) on the CUDA path against
the FP64 oracle at the same iteration count, 2D and 3D, real and complex, and
relaxed-FISTA steps with tv_kind = 1 against the oracle's steps."""
import numpy as np
import pytest

from oracle import fista, grad, prox
from paper_1708_01663_gb300 import synth
from tests.gpu_util import c64, make, rel
from tests.test_gpu_3d import make3

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [64, 37])
@pytest.mark.parametrize("complex_f", [False, True])
def test_tv_aniso_2d(n, complex_f):
    ctx, _ = make(n, 2, 4, 0.75 * n / 8 + 1.0, complex_f=complex_f)
    z = synth.ellipse_phantom(n, 4, (0.0, 1.0), 5, 0.2) + 0.1 * synth.random_field(6, (n, n))
    x = np.empty((n, n), np.complex64)
    lam, iters = 0.05, 30
    ctx.tv_prox(c64(z), x, lam, iters, 0.0, 0.9, 0.0, 0.15, aniso=True)
    zc = c64(z).astype(np.complex128)
    ref = prox.prox_R_aniso(zc, lam, iters, (0.0, 0.9), (0.0, 0.15) if complex_f else None)
    assert np.abs(x - ref).max() < 2e-5
    ctx.tv_prox(c64(z), x, 0.0, iters, 0.0, 0.9, 0.0, 0.15, aniso=True)
    assert np.array_equal(x.real, np.clip(c64(z).real, 0.0, 0.9))


@pytest.mark.parametrize("n", [16, 21])
def test_tv_aniso_3d(n):
    ctx, _ = make3(n, 1, complex_f=True)
    z = synth.sphere_phantom(n, 4, (0.0, 1.0), 5, 0.2) + 0.1 * synth.random_field(6, (n, n, n))
    x = np.empty((n, n, n), np.complex64)
    ctx.tv_prox(c64(z), x, 0.05, 25, 0.0, 0.9, 0.0, 0.15, aniso=True)
    ref = prox.prox_R_aniso(c64(z).astype(np.complex128), 0.05, 25, (0.0, 0.9), (0.0, 0.15))
    assert np.abs(x - ref).max() < 2e-5


def _aniso_fista(prob, y, f0, gamma, tau, alpha, K, tv_iters):
    """The oracle's relaxed FISTA with the anisotropic prox in place of FGP."""
    import math
    f_prev = np.array(f0, dtype=np.complex128)
    s = f_prev.copy()
    t, hist = 1.0, []
    for _ in range(K):
        D, g = grad.data_and_grad(prob, s, y, tol=1e-11)
        f = prox.prox_R_aniso(s - gamma * g.real, gamma * tau, tv_iters)
        tn = (math.sqrt(4 * t * t + 1) + 1) / 2
        s = f + alpha * ((t - 1) / tn) * (f - f_prev)
        f_prev, t = f, tn
        hist.append(D)
    return f_prev, hist


def test_relaxed_fista_aniso_steps():
    cfg = synth.CONFIGS["c1"]
    n, T, M = cfg["n"], cfg["T"], cfg["M"]
    ctx, prob = make(n, T, M, cfg["rx_radius"])
    f_true = synth.ellipse_phantom(n, cfg["shapes"], cfg["contrast"], cfg["seed"])
    _, y, _, _ = grad.forward(prob, f_true, tol=1e-12)
    gamma = 1.0 / grad.born_hessian_norm(prob)
    K, tau = 6, 3e-3
    ref, hist = _aniso_fista(prob, y, np.zeros((n, n)), gamma, tau, cfg["alpha"], K, 20)
    f = np.zeros((n, n), np.complex64)
    s = np.zeros((n, n), np.complex64)
    st = ctx.new_state(f, s, cfg["alpha"], gamma, tau, 20, 0.0, 2.0, tv_kind=1)
    Ds = []
    for _ in range(K):
        ctx.step(st, c64(y), tol=1e-6, max_iter=3000, x0_mode=0)
        Ds.append(st.D)
    assert rel(Ds, hist) < 1e-3
    assert rel(f, ref) <= 1e-3
