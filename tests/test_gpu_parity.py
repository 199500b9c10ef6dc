"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (complex64 arithmetic with FP64 reductions):
  tables (FP64 -> c64 rounding)                   rel-L2 <= 1e-6
  one FFT matvec A x / A^H x (FP32 FFTs, P<=512)   rel-L2 <= 2e-5
  fields at solver tol 1e-6 vs oracle at 1e-12     rel-L2 <= 1e-4   (spec field bar)
  sensing GEMMs                                    rel-L2 <= 1e-5
  gradient (two solves, one extra convolution)     rel-L2 <= 5e-4
  FGP prox, same iteration count                   max-abs <= 2e-5
  relaxed FISTA reconstruction after K steps       rel-L2 <= 1e-3   (spec reconstruction bar)
"""
import numpy as np
import pytest

from oracle import fista, grad, model, prox, solve
from paper_1708_01663_gb300 import synth
from tests.gpu_util import c64, make, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,pad", [(64, 0), (40, 0), (100, 0), (96, 512), (256, 0)])
def test_tables(n, pad):
    ctx, prob = make(n, 3, 16, 0.75 * n / 8 + 1.0, pad=pad)
    gh = np.empty((ctx.P, ctx.P), np.complex64)
    ctx.green_spectrum(gh)
    assert rel(gh, prob.ghat) < 1e-6
    H = np.empty((ctx.M, ctx.N), np.complex64)
    ctx.sensing_matrix(H)
    assert rel(H, prob.H) < 1e-6
    u = np.empty((ctx.T, n, n), np.complex64)
    ctx.incident(u)
    assert rel(u, prob.u_in) < 1e-6


@pytest.mark.parametrize("n", [64, 40, 100, 256])
@pytest.mark.parametrize("adjoint", [False, True])
def test_apply_A(n, adjoint):
    ctx, prob = make(n, 3, 8, 0.75 * n / 8 + 1.0)
    f = synth.ellipse_phantom(n, 4, (0.0, 0.8), 7, imag=0.05)
    x = synth.random_field(8, (3, n, n))
    y = np.empty((3, n, n), np.complex64)
    ctx.apply_A(c64(f), c64(x), y, adjoint=adjoint)
    op = prob.AH if adjoint else prob.A
    for t in range(3):
        assert rel(y[t], op(f, x[t])) < 2e-5


def test_apply_A_two_vectors_of_more():
    # nvec < T: only the first nvec transmitter slots are used
    ctx, prob = make(64, 5, 8, 6.0)
    f = synth.ellipse_phantom(64, 3, (0.0, 0.5), 2)
    x = synth.random_field(3, (2, 64, 64))
    y = np.empty((2, 64, 64), np.complex64)
    ctx.apply_A(c64(f), c64(x), y)
    assert rel(y[1], prob.A(f, x[1])) < 2e-5


def _forward_parity(n, T, M, contrast, imag, seed, tol=1e-6):
    ctx, prob = make(n, T, M, 0.75 * n / 8 + 1.5)
    f = synth.ellipse_phantom(n, 3, contrast, seed, imag)
    u = np.empty((T, n, n), np.complex64)
    y = np.empty((T, M), np.complex64)
    st, info = ctx.forward(c64(f), u_out=u, y_out=y, tol=tol, max_iter=3000)
    ref, its, res = solve.solve_fields(prob, f, prob.u_in, tol=1e-12)
    yref = prob.sense(f, ref)
    return u, y, ref, yref, info


def test_forward_c1_sizes():
    cfg = synth.CONFIGS["c1"]
    u, y, ref, yref, info = _forward_parity(cfg["n"], cfg["T"], cfg["M"], cfg["contrast"], 0.0, cfg["seed"])
    assert info.resid_max <= 1e-6
    assert rel(u, ref) <= 1e-4
    assert rel(y, yref) <= 1e-4


@pytest.mark.parametrize("n,T", [(40, 3), (100, 5)])
def test_forward_ragged_high_contrast(n, T):
    u, y, ref, yref, info = _forward_parity(n, T, 24, (0.3, 0.9), 0.05, 77)
    for t in range(T):
        assert rel(u[t], ref[t]) <= 1e-4, (t, rel(u[t], ref[t]))
    assert rel(y, yref) <= 1e-4


def test_forward_zero_contrast_is_incident_field():
    ctx, prob = make(64, 4, 8, 6.0)
    u = np.empty((4, 64, 64), np.complex64)
    y = np.empty((4, 8), np.complex64)
    st, info = ctx.forward(np.zeros((64, 64), np.complex64), u_out=u, y_out=y, tol=1e-6)
    assert info.iters_max == 0
    assert rel(u, prob.u_in) < 1e-6
    assert np.abs(y).max() == 0.0


def test_forward_warm_start_keeps_solution():
    ctx, prob = make(64, 4, 8, 6.0)
    f = c64(synth.ellipse_phantom(64, 3, (0.0, 0.3), 4))
    u1 = np.empty((4, 64, 64), np.complex64)
    ctx.forward(f, u_out=u1, tol=1e-6)
    st, info = ctx.forward(f, u_out=u1, tol=1e-6, x0_mode=2)
    assert info.iters_max == 0          # previous solution already meets tol
    st, info = ctx.forward(f, x0=u1, u_out=u1, tol=1e-6, x0_mode=1)
    assert info.iters_max == 0


# tensor cores (even sizes, T <= 128: 40 x 2 and 6 x 2 columns) and the FP32 fallback (odd receiver count,
# odd field length, T > 128)
@pytest.mark.parametrize("n,T,M", [(64, 6, 40), (40, 3, 24), (64, 6, 41), (63, 6, 40), (32, 130, 16)])
def test_sense_and_adjoint(n, T, M):
    ctx, prob = make(n, T, M, 6.5)
    f = synth.ellipse_phantom(n, 3, (0.0, 0.5), 9, imag=0.02)
    u = synth.random_field(10, (T, n, n))
    Z = np.empty((T, M), np.complex64)
    ctx.sense(c64(f), c64(u), Z)
    assert rel(Z, prob.sense(f, u)) < 1e-5
    w = synth.random_field(11, (T, M))
    z = np.empty((T, n, n), np.complex64)
    b = np.empty((T, n, n), np.complex64)
    ctx.sense_adjoint(c64(f), c64(w), z, b)
    zref = (w @ np.conj(prob.H)).reshape(T, n, n)
    assert rel(z, zref) < 1e-5
    assert rel(b, np.conj(f)[None] * zref) < 1e-5


@pytest.mark.parametrize("complex_f", [False, True])
def test_gradient(complex_f):
    n, T, M = 48, 4, 24
    ctx, prob = make(n, T, M, 5.0, complex_f=complex_f)
    imag = 0.03 if complex_f else 0.0
    f = synth.ellipse_phantom(n, 3, (0.1, 0.5), 12, imag)
    f_true = synth.ellipse_phantom(n, 3, (0.1, 0.6), 13, imag)
    _, y, _, _ = grad.forward(prob, f_true, tol=1e-12)
    D_ref, g_ref = grad.data_and_grad(prob, f, y, tol=1e-12)
    g = np.empty((n, n), np.complex64)
    D, st, info = ctx.grad(c64(f), c64(y), g, tol=1e-6, max_iter=3000)
    assert abs(D - D_ref) / D_ref < 1e-4
    if complex_f:
        assert rel(g, g_ref) < 5e-4
    else:
        assert rel(g.real, g_ref.real) < 5e-4


@pytest.mark.parametrize("n,P", [(100, 256), (64, 128)])
def test_forward_two_stage_2d(n, P):
    """Forward solves through the two-stage column kernels at P = 256 (16 x 16) and
    P = 128 (16 x 8) in 2D reach the oracle's fields."""
    ctx, prob = make(n, 3, 16, 0.75 * n / 8 + 1.5)
    assert ctx.P == P
    ctx.set_cols_cta(16)
    f = synth.ellipse_phantom(n, 3, (0.1, 0.6), 41, 0.03)
    u = np.empty((3, n, n), np.complex64)
    st, info = ctx.forward(c64(f), u_out=u, tol=1e-6, max_iter=3000)
    ref, _, _ = solve.solve_fields(prob, f, prob.u_in, tol=1e-12)
    assert info.resid_max <= 1e-6
    assert rel(u, ref) <= 1e-4


@pytest.mark.parametrize("shape", [512, 16, 8])
def test_gradient_p512_shapes(shape):
    """D and the gradient at P = 512 (n = 130: most of each padded row and column
    empty) with the three-stage kernels, the two-stage column kernel and the
    one-kernel cluster pass (shape 8: an 8-CTA cluster per transmitter, the
    padded field in distributed shared memory); exercises every prologue,
    epilogue and dot set of the solves plus the G^H v + z epilogue of the
    gradient."""
    n, T, M = 130, 2, 24
    ctx, prob = make(n, T, M, 0.75 * n / 8 + 1.5, complex_f=True)
    assert ctx.P == 512
    ctx.set_cols_cta(shape)
    f = synth.ellipse_phantom(n, 3, (0.05, 0.3), 31, 0.02)
    f_true = synth.ellipse_phantom(n, 3, (0.05, 0.35), 32, 0.02)
    _, y, _, _ = grad.forward(prob, f_true, tol=1e-12)
    D_ref, g_ref = grad.data_and_grad(prob, f, y, tol=1e-12)
    g = np.empty((n, n), np.complex64)
    D, st, info = ctx.grad(c64(f), c64(y), g, tol=1e-6, max_iter=3000)
    assert abs(D - D_ref) / D_ref < 1e-4
    assert rel(g, g_ref) < 5e-4


@pytest.mark.parametrize("complex_f", [False, True])
def test_tv_prox(complex_f):
    n = 64
    ctx, _ = make(n, 2, 4, 6.0, complex_f=complex_f)
    z = synth.ellipse_phantom(n, 4, (0.0, 1.0), 5, 0.2) + 0.1 * synth.random_field(6, (n, n))
    x = np.empty((n, n), np.complex64)
    lam, iters = 0.05, 20
    ctx.tv_prox(c64(z), x, lam, iters, 0.0, 0.9, 0.0, 0.15)
    ref = prox.prox_R(c64(z).astype(np.complex128), lam, iters, (0.0, 0.9), (0.0, 0.15) if complex_f else None)
    assert np.abs(x - ref).max() < 2e-5
    # zero weight is the clamp
    ctx.tv_prox(c64(z), x, 0.0, iters, 0.0, 0.9, 0.0, 0.15)
    zc = c64(z)
    assert np.array_equal(x.real, np.clip(zc.real, 0.0, 0.9))


def _c1_problem():
    cfg = synth.CONFIGS["c1"]
    n, T, M = cfg["n"], cfg["T"], cfg["M"]
    ctx, prob = make(n, T, M, cfg["rx_radius"])
    f_true = synth.ellipse_phantom(n, cfg["shapes"], cfg["contrast"], cfg["seed"])
    _, y_clean, _, _ = grad.forward(prob, f_true, tol=1e-12)
    e = synth.complex_noise(cfg["seed"] + 100, y_clean.shape)
    sigma = np.linalg.norm(y_clean) * 10 ** (-cfg["snr_db"] / 20) / np.sqrt(y_clean.size)
    y = y_clean + sigma * e
    gamma = 1.0 / grad.born_hessian_norm(prob)
    return cfg, ctx, prob, f_true, y, gamma


def _fista_parity(alpha, K):
    cfg, ctx, prob, f_true, y, gamma = _c1_problem()
    n = cfg["n"]
    ref, hist = fista.relaxed_fista(prob, y, np.zeros((n, n)), gamma, cfg["tau"], alpha, K,
                                    cfg["tv_iters"], tol=1e-11)
    f = np.zeros((n, n), np.complex64)
    s = np.zeros((n, n), np.complex64)
    st = ctx.new_state(f, s, alpha, gamma, cfg["tau"], cfg["tv_iters"], 0.0, 2.0)
    Ds = []
    for _ in range(K):
        ctx.step(st, c64(y), tol=1e-6, max_iter=3000)
        Ds.append(st.D)
    assert rel(Ds, hist) < 1e-3
    assert rel(f, ref) <= 1e-3
    return f, f_true, hist


def test_relaxed_fista_c1_reconstruction():
    cfg = synth.CONFIGS["c1"]
    f, f_true, _ = _fista_parity(cfg["alpha"], cfg["outer"])
    assert fista.recon_snr_db(f, f_true) > 3.0


@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_relaxed_fista_ista_and_fista_ends(alpha):
    """The two ends of the relaxation (Sec. III-A): alpha = 0 is ISTA (no momentum), alpha = 1 plain
    FISTA; 10 steps of each on the C1 workload against the oracle's trajectory."""
    _fista_parity(alpha, 10)


def test_solve_iterations_and_cols_cta():
    ctx, prob = make(64, 5, 8, 6.0)
    assert len(ctx.solve_iterations()) == 0
    f = c64(synth.ellipse_phantom(64, 3, (0.0, 0.5), 14))
    u = np.empty((5, 64, 64), np.complex64)
    st, info = ctx.forward(f, u_out=u, tol=1e-6)
    it = ctx.solve_iterations()
    assert len(it) == 5 and it.max() == info.iters_max and abs(it.mean() - info.iters_mean) < 1e-12
    x = synth.random_field(15, (5, 64, 64))
    y512 = np.empty((5, 64, 64), np.complex64)
    y256 = np.empty((5, 64, 64), np.complex64)
    ctx.set_cols_cta(512)
    ctx.apply_A(f, c64(x), y512)
    ctx.set_cols_cta(256)
    ctx.apply_A(f, c64(x), y256)
    assert rel(y256, y512) < 1e-6
    for t in range(5):
        assert rel(y256[t], prob.A(f.astype(np.complex128), x[t])) < 2e-5
    # the re-captured solver graphs use the new shape and still converge to the same fields
    u2 = np.empty_like(u)
    ctx.forward(f, u_out=u2, tol=1e-6)
    assert rel(u2, u) < 1e-5
    with pytest.raises(Exception):
        ctx.set_cols_cta(128)
    small, _ = make(20, 2, 8, 3.0)
    assert small.P == 64
    with pytest.raises(Exception):
        small.set_cols_cta(16)  # no two-stage plan at P = 64


@pytest.mark.parametrize("n,pad,P", [(256, 0, 512), (96, 512, 512), (100, 0, 256), (40, 256, 256), (64, 0, 128),
                                     (33, 128, 128)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_column_shapes(n, pad, P, adjoint):
    """Every column-kernel shape (the three-stage kernel at 512 and 256 threads,
    the two-stage kernel: 32 x 16 at P = 512, 16 x 16 at 256, 16 x 8 at 128;
    at P = 512 also the one-kernel cluster pass)
    against the oracle's A / A^H; a padded n leaves most of each column empty
    (ragged rows and columns)."""
    ctx, prob = make(n, 3, 8, 0.75 * n / 8 + 1.0, pad=pad)
    assert ctx.P == P
    f = synth.ellipse_phantom(n, 4, (0.0, 0.8), 7, imag=0.05)
    x = synth.random_field(8, (3, n, n))
    op = prob.AH if adjoint else prob.A
    ys = {}
    for shape in ((512, 256, 16, 8) if P == 512 else (512, 256, 16)):
        ctx.set_cols_cta(shape)
        y = np.empty((3, n, n), np.complex64)
        ctx.apply_A(c64(f), c64(x), y, adjoint=adjoint)
        for t in range(3):
            assert rel(y[t], op(f, x[t])) < 2e-5, shape
        ys[shape] = y
    assert rel(ys[16], ys[512]) < 1e-5


def test_two_stage_shape_solves_and_autotunes():
    """Forward solves with the two-stage column kernel converge to the oracle's
    fields, and the autotuner may pick any of the three shapes at P = 512."""
    n = 256
    ctx, prob = make(n, 2, 8, 0.75 * n / 8 + 1.5)
    f = synth.ellipse_phantom(n, 5, (0.0, 0.3), 21)
    ctx.set_cols_cta(16)
    u = np.empty((2, n, n), np.complex64)
    st, info = ctx.forward(c64(f), u_out=u, tol=1e-6, max_iter=3000)
    assert info.resid_max <= 1e-6
    ref, its, res = solve.solve_fields(prob, f, prob.u_in, tol=1e-12)
    assert rel(u, ref) < 1e-4
    assert ctx.autotune(reps=2) in (512, 256, 16, 8)
    with pytest.raises(Exception):
        make(64, 1, 8, 6.0, complex_f=False)[0].set_cols_cta(8)


@pytest.mark.parametrize("n,T", [(256, 5), (64, 7)])
def test_tx_chunks_keep_results(n, T):
    """A convolution pass split into transmitter chunks (each chunk's whole row / column / row chain
    before the next, all reusing the start of the intermediate) gives the same A x, A^H x and solved
    fields as one launch over all transmitters, and matches the oracle."""
    ctx, prob = make(n, T, 8, 0.75 * n / 8 + 1.0, complex_f=True)
    f = synth.ellipse_phantom(n, 4, (0.0, 0.8), 7, imag=0.05)
    x = synth.random_field(8, (T, n, n))
    ref = {}
    for chunk in (0, 2, 3, T + 1):
        ctx.set_tx_chunk(chunk)
        assert ctx.tuning()[1] == chunk
        for adjoint in (False, True):
            y = np.empty((T, n, n), np.complex64)
            ctx.apply_A(c64(f), c64(x), y, adjoint=adjoint)
            if chunk == 0:
                ref[adjoint] = y
                op = prob.AH if adjoint else prob.A
                for t in (0, T - 1):
                    assert rel(y[t], op(f, x[t])) < 2e-5
            else:
                assert rel(y, ref[adjoint]) < 1e-6, (chunk, adjoint)
        u = np.empty((T, n, n), np.complex64)
        st, info = ctx.forward(c64(f), u_out=u, tol=1e-6, max_iter=3000)
        assert info.resid_max <= 1e-6
        if chunk == 0:
            ref["u"] = u
        else:
            assert rel(u, ref["u"]) < 1e-5


def test_device_side_solve_loop_matches_host_loop():
    """The whole solve as one graph launch (a WHILE node over chunks of BiCGSTAB iterations, ended by
    a device-side condition kernel) gives the fields, iteration counts and residuals of the
    host-driven chunk loop, and the oracle's fields (Eq. 13)."""
    n, T = 64, 5
    ctx, prob = make(n, T, 8, 6.0, complex_f=True)
    f = c64(synth.ellipse_phantom(n, 4, (0.0, 0.8), 41, 0.05))
    res = {}
    for mode in (False, True):
        ctx.set_solve_loop(mode)
        u = np.empty((T, n, n), np.complex64)
        st, info = ctx.forward(f, u_out=u, tol=1e-6, max_iter=3000)
        assert info.resid_max <= 1e-6
        res[mode] = (u, ctx.solve_iterations().tolist())
    assert res[True][1] == res[False][1]
    assert rel(res[True][0], res[False][0]) < 1e-6
    ref, _, _ = solve.solve_fields(prob, f.astype(np.complex128), prob.u_in, tol=1e-12)
    assert rel(res[True][0], ref) < 1e-4
