"""3D scalar model (Eq. 1 with d = 3, Appendix A grid) on the CUDA path vs the
FP64 oracle, through the C ABI.  Same bars as the 2D parity tests:
  tables                          rel-L2 <= 1e-6
  one matvec A x / A^H x          rel-L2 <= 2e-5
  fields at tol 1e-6              rel-L2 <= 1e-4
  gradient                        rel-L2 <= 5e-4
  FGP prox (same iterations)      max-abs <= 2e-5
  relaxed FISTA after K steps     rel-L2 <= 1e-3
Sizes span several row tiles with a ragged tail (n = 33: 1089 x rows over
16-row tiles) and both FFT sides used in 3D (P = 64, 128).
"""
import numpy as np
import pytest

from oracle import fista, grad, model, prox, solve
from paper_1708_01663_gb300 import build, cisor, synth
from tests.gpu_util import c64, rel

pytestmark = pytest.mark.gpu

DELTA = 1.0 / 6


def _dirs(T):
    return synth.hemisphere_directions()[:T]


def _rx(n, M=64):
    side = int(np.sqrt(M))
    return synth.planar_receivers(side, 0.5, 0.6 * n * DELTA + 1.0)


def make3(n, T, M=64, pad=0, complex_f=False):
    build.build()
    dirs, rx = _dirs(T), _rx(n, M)
    ctx = cisor.Cisor(n, DELTA, dirs, rx, complex_f=complex_f, pad=pad, dim=3)
    prob = model.Problem(n, DELTA, dirs, rx, P=ctx.P, dim=3)
    return ctx, prob


@pytest.mark.parametrize("n,pad", [(16, 0), (33, 0), (20, 128)])
def test_tables_3d(n, pad):
    ctx, prob = make3(n, 3, pad=pad)
    P = 64
    while P < 2 * n - 1:
        P *= 2
    assert ctx.N == n ** 3 and ctx.P == (pad or P)
    gh = np.empty((ctx.P,) * 3, np.complex64)
    ctx.green_spectrum(gh)
    assert rel(gh, prob.ghat) < 1e-6
    H = np.empty((ctx.M, ctx.N), np.complex64)
    ctx.sensing_matrix(H)
    assert rel(H, prob.H) < 1e-6
    u = np.empty((ctx.T, n, n, n), np.complex64)
    ctx.incident(u)
    assert rel(u, prob.u_in) < 1e-6


@pytest.mark.parametrize("n,pad", [(16, 0), (33, 0), (20, 128)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_apply_A_3d(n, pad, adjoint):
    ctx, prob = make3(n, 3, pad=pad)
    f = synth.sphere_phantom(n, 4, (0.0, 0.6), 7, imag=0.05)
    x = synth.random_field(8, (3, n, n, n))
    y = np.empty((3, n, n, n), np.complex64)
    ctx.apply_A(c64(f), c64(x), y, adjoint=adjoint)
    op = prob.AH if adjoint else prob.A
    for t in range(3):
        assert rel(y[t], op(f, x[t])) < 2e-5


@pytest.mark.parametrize("n,pad", [(33, 0), (20, 128), (40, 256)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_apply_A_3d_two_stage(n, pad, adjoint):
    """The two-stage column kernels (16 x 8 at P = 128, 16 x 16 at P = 256) in all
    three 3D modes (y forward, z spectrum product, y inverse) against the oracle."""
    ctx, prob = make3(n, 3, pad=pad)
    ctx.set_cols_cta(16)
    f = synth.sphere_phantom(n, 4, (0.0, 0.6), 7, imag=0.05)
    x = synth.random_field(8, (3, n, n, n))
    y = np.empty((3, n, n, n), np.complex64)
    ctx.apply_A(c64(f), c64(x), y, adjoint=adjoint)
    op = prob.AH if adjoint else prob.A
    for t in range(3):
        assert rel(y[t], op(f, x[t])) < 2e-5


def test_forward_3d_two_stage():
    ctx, prob = make3(33, 2)
    ctx.set_cols_cta(16)
    f = synth.sphere_phantom(33, 4, (0.1, 0.5), 21, imag=0.02)
    u = np.empty((2, 33, 33, 33), np.complex64)
    st, info = ctx.forward(c64(f), u_out=u, tol=1e-6, max_iter=3000)
    ref, _, _ = solve.solve_fields(prob, f, prob.u_in, tol=1e-12)
    assert info.resid_max <= 1e-6
    assert rel(u, ref) <= 1e-4


@pytest.mark.parametrize("n,T", [(16, 4), (33, 2)])
def test_forward_3d(n, T):
    ctx, prob = make3(n, T)
    f = synth.sphere_phantom(n, 4, (0.1, 0.5), 21, imag=0.02)
    u = np.empty((T, n, n, n), np.complex64)
    y = np.empty((T, ctx.M), np.complex64)
    st, info = ctx.forward(c64(f), u_out=u, y_out=y, tol=1e-6, max_iter=3000)
    ref, _, _ = solve.solve_fields(prob, f, prob.u_in, tol=1e-12)
    assert info.resid_max <= 1e-6
    for t in range(T):
        assert rel(u[t], ref[t]) <= 1e-4
    assert rel(y, prob.sense(f, ref)) <= 1e-4


def test_forward_3d_zero_contrast():
    ctx, prob = make3(16, 2)
    u = np.empty((2, 16, 16, 16), np.complex64)
    st, info = ctx.forward(np.zeros((16, 16, 16), np.complex64), u_out=u, tol=1e-6)
    assert info.iters_max == 0
    assert rel(u, prob.u_in) < 1e-6


@pytest.mark.parametrize("complex_f", [False, True])
def test_gradient_3d(complex_f):
    n, T = 16, 3
    ctx, prob = make3(n, T, complex_f=complex_f)
    imag = 0.03 if complex_f else 0.0
    f = synth.sphere_phantom(n, 3, (0.1, 0.4), 12, imag)
    f_true = synth.sphere_phantom(n, 3, (0.1, 0.5), 13, imag)
    _, y, _, _ = grad.forward(prob, f_true, tol=1e-12)
    D_ref, g_ref = grad.data_and_grad(prob, f, y, tol=1e-12)
    g = np.empty((n, n, n), np.complex64)
    D, st, info = ctx.grad(c64(f), c64(y), g, tol=1e-6, max_iter=3000)
    assert abs(D - D_ref) / D_ref < 1e-4
    if complex_f:
        assert rel(g, g_ref) < 5e-4
    else:
        assert rel(g.real, g_ref.real) < 5e-4


@pytest.mark.parametrize("n", [16, 33])
@pytest.mark.parametrize("complex_f", [False, True])
def test_tv_prox_3d(n, complex_f):
    ctx, _ = make3(n, 1, complex_f=complex_f)
    z = synth.sphere_phantom(n, 4, (0.0, 1.0), 5, 0.2) + 0.1 * synth.random_field(6, (n, n, n))
    x = np.empty((n, n, n), np.complex64)
    lam, iters = 0.05, 20
    ctx.tv_prox(c64(z), x, lam, iters, 0.0, 0.9, 0.0, 0.15)
    ref = prox.prox_R(c64(z).astype(np.complex128), lam, iters, (0.0, 0.9), (0.0, 0.15) if complex_f else None)
    assert np.abs(x - ref).max() < 2e-5


def test_relaxed_fista_3d():
    n, T = 16, 6
    ctx, prob = make3(n, T)
    f_true = synth.sphere_phantom(n, 3, (0.0, 0.3), 31)
    _, y, _, _ = grad.forward(prob, f_true, tol=1e-12)
    gamma = 1.0 / grad.born_hessian_norm(prob)
    K, tau, alpha, tv_iters = 6, 1e-3, 0.96, 10
    ref, hist = fista.relaxed_fista(prob, y, np.zeros((n, n, n)), gamma, tau, alpha, K, tv_iters, tol=1e-11)
    f = np.zeros((n, n, n), np.complex64)
    s = np.zeros((n, n, n), np.complex64)
    st = ctx.new_state(f, s, alpha, gamma, tau, tv_iters, 0.0, 2.0)
    Ds = []
    for _ in range(K):
        ctx.step(st, c64(y), tol=1e-6, max_iter=3000)
        Ds.append(st.D)
    assert rel(Ds, hist) < 1e-3
    assert rel(f, ref) <= 1e-3


def test_c3_full_size_sampled():
    """The 64^3, 48-transmitter, 1024-receiver workload in the bench's launch
    configuration: tables against the oracle (spectrum in full, H rows and
    incident fields sampled); forward fields checked on sampled transmitters
    through the oracle's FP64 operator (true residual) and its sensing."""
    cfg, f, dirs, rx = synth.make_inputs("c3")
    n, T = cfg["n"], cfg["T"]
    build.build()
    ctx = cisor.Cisor(n, cfg["delta"], dirs, rx, dim=3)
    ctx.autotune()
    assert (ctx.P, ctx.N, ctx.T, ctx.M) == (128, n ** 3, T, 1024)
    k, kb = model.wavenumbers(1.0)
    gh = np.empty((128,) * 3, np.complex64)
    ctx.green_spectrum(gh)
    assert rel(gh, model.green_spectrum(n, 128, cfg["delta"], k, kb, dim=3)) < 1e-6
    H = np.empty((ctx.M, ctx.N), np.complex64)
    ctx.sensing_matrix(H)
    rows = [0, 517, 1023]
    assert rel(H[rows], model.sensing_matrix(rx[rows], n, cfg["delta"], k, kb)) < 1e-6
    u = np.empty((T, n, n, n), np.complex64)
    y = np.empty((T, ctx.M), np.complex64)
    st, info = ctx.forward(c64(f), u_out=u, y_out=y, tol=1e-4, max_iter=2000)
    assert info.n_not_converged == 0 and info.resid_max <= 1e-4
    ghat = model.green_spectrum(n, 128, cfg["delta"], k, kb, dim=3)
    ts = [0, 29, 47]
    for t in ts:
        uin = model.plane_waves_3d(dirs[t:t + 1], n, cfg["delta"], kb)[0]
        ut = u[t].astype(np.complex128)
        res = np.linalg.norm(uin - model.apply_A(f, ut, ghat)) / np.linalg.norm(uin)
        assert res <= 2e-4, (t, res)
    # Z_t = H diag(u_t) f over receiver chunks (the dense H is 4 GB in FP64)
    V = np.stack([(f * u[t].astype(np.complex128)).ravel() for t in ts], axis=1)
    Zref = np.concatenate([model.sensing_matrix(rx[m:m + 64], n, cfg["delta"], k, kb) @ V
                           for m in range(0, ctx.M, 64)])
    assert rel(y[ts].T, Zref) < 1e-5


def test_tx_chunks_keep_results_3d():
    """Transmitter chunks in the five-kernel 3D pass (every chunk reusing the start of the
    [chunk, n, P, P] intermediate) give the same A x and fields as one launch, and the oracle's A x."""
    n, T = 24, 5
    ctx, prob = make3(n, T)
    f = synth.sphere_phantom(n, 3, (0.0, 0.3), 8)
    x = synth.random_field(9, (T, n, n, n))
    ys, us = [], []
    for chunk in (0, 2):
        ctx.set_tx_chunk(chunk)
        y = np.empty((T, n, n, n), np.complex64)
        ctx.apply_A(c64(f), c64(x), y)
        u = np.empty((T, n, n, n), np.complex64)
        ctx.forward(c64(f), u_out=u, tol=1e-6, max_iter=3000)
        ys.append(y)
        us.append(u)
    for t in (0, T - 1):
        assert rel(ys[0][t], prob.A(f, x[t])) < 2e-5
    assert rel(ys[1], ys[0]) < 1e-6
    assert rel(us[1], us[0]) < 1e-5
