"""3D vectorial model (appendix) on the CUDA path vs the FP64 oracle: dyadic
sensing table and polarised incident fields, A / A^H (convolution plus the
finite-difference grad-div stencil), field solves, the gradient, relaxed-FISTA
steps, and the full 32^3 C7 workload sampled.  Bars as in the scalar tests."""
import numpy as np
import pytest

from oracle import fista, vector
from paper_1708_01663_gb300 import build, cisor, synth
from tests.gpu_util import c64, rel

pytestmark = pytest.mark.gpu

DELTA = 1.0 / 10


def _geom(n, T, M=12):
    tx = synth.polarised_hemisphere(3, 4)[:T]
    phi = 2 * np.pi * np.arange(M) / M
    r = 0.5 * n * DELTA + 1.5
    rx = np.stack([r * np.cos(phi), r * np.sin(phi), 0.4 * np.sin(3 * phi)], 1)
    return tx, rx


def make_vec(n, T, M=12, complex_f=False):
    build.build()
    tx, rx = _geom(n, T, M)
    ctx = cisor.Cisor(n, DELTA, tx, rx, dim=3, vectorial=True, complex_f=complex_f)
    prob = vector.VectorProblem(n, DELTA, tx[:, :3], tx[:, 3:], rx, P=ctx.P)
    return ctx, prob


@pytest.mark.parametrize("n", [8, 13])
def test_vector_tables(n):
    ctx, prob = make_vec(n, 3)
    assert ctx.Nf == 3 * n ** 3
    H = np.empty((ctx.M, ctx.Nf), np.complex64)
    ctx.sensing_matrix(H)
    assert rel(H, prob.H) < 1e-6
    u = np.empty((ctx.T, 3, n, n, n), np.complex64)
    ctx.incident(u)
    assert rel(u, prob.u_in) < 1e-6


@pytest.mark.parametrize("n", [16, 13])
@pytest.mark.parametrize("adjoint", [False, True])
def test_vector_apply_A(n, adjoint):
    ctx, prob = make_vec(n, 3)
    f = synth.sphere_phantom(n, 3, (0.2, 0.9), 7, imag=0.05)
    x = synth.random_field(8, (3, 3, n, n, n))
    y = np.empty((3, 3, n, n, n), np.complex64)
    ctx.apply_A(c64(f), c64(x), y, adjoint=adjoint)
    op = prob.AH if adjoint else prob.A
    for t in range(3):
        assert rel(y[t], op(f, x[t])) < 2e-5


def test_vector_forward():
    n, T = 12, 3
    ctx, prob = make_vec(n, T)
    f = synth.sphere_phantom(n, 3, (0.3, 1.0), 21, imag=0.02)
    u = np.empty((T, 3, n, n, n), np.complex64)
    y = np.empty((T, ctx.M), np.complex64)
    st, info = ctx.forward(c64(f), u_out=u, y_out=y, tol=1e-6, max_iter=3000)
    ref = vector.solve_fields(prob, f, prob.u_in, tol=1e-12)
    assert info.resid_max <= 1e-6
    for t in range(T):
        assert rel(u[t], ref[t]) <= 1e-4
    assert rel(y, prob.sense(f, ref)) <= 1e-4


@pytest.mark.parametrize("complex_f", [False, True])
def test_vector_gradient(complex_f):
    n, T = 10, 2
    ctx, prob = make_vec(n, T, complex_f=complex_f)
    imag = 0.03 if complex_f else 0.0
    f = synth.sphere_phantom(n, 3, (0.1, 0.5), 12, imag)
    ft = synth.sphere_phantom(n, 3, (0.2, 0.7), 13, imag)
    y = prob.sense(ft, vector.solve_fields(prob, ft, prob.u_in, tol=1e-12))
    D_ref, g_ref = vector.data_and_grad(prob, f, y, tol=1e-12)
    g = np.empty((n, n, n), np.complex64)
    D, st, info = ctx.grad(c64(f), c64(y), g, tol=1e-6, max_iter=3000)
    assert abs(D - D_ref) / D_ref < 1e-4
    assert rel(g if complex_f else g.real, g_ref if complex_f else g_ref.real) < 5e-4


def test_vector_fista_steps():
    n, T = 12, 4
    ctx, prob = make_vec(n, T)
    ft = synth.sphere_phantom(n, 2, (0.2, 0.6), 31)
    y = prob.sense(ft, vector.solve_fields(prob, ft, prob.u_in, tol=1e-12))
    s0 = np.zeros((n, n, n))
    _, g0 = vector.data_and_grad(prob, s0, y, tol=1e-12)
    gamma = 0.2 * float(np.linalg.norm(ft)) / float(np.linalg.norm(g0.real))
    K, tau, alpha, tv_iters = 4, 1e-3, 0.96, 10

    def gfn(s, state):
        return vector.data_and_grad(prob, s, y, tol=1e-11)

    ref, hist = fista.relaxed_fista(prob, None, s0, gamma, tau, alpha, K, tv_iters, grad_fn=gfn)
    f = np.zeros((n, n, n), np.complex64)
    s = np.zeros((n, n, n), np.complex64)
    st = ctx.new_state(f, s, alpha, gamma, tau, tv_iters, 0.0, 2.0)
    Ds = []
    for _ in range(K):
        ctx.step(st, c64(y), tol=1e-6, max_iter=3000, x0_mode=0)
        Ds.append(st.D)
    assert rel(Ds, hist) < 1e-3
    assert rel(f, ref) <= 1e-3


def test_c7_full_size_sampled():
    """The 32^3, 81-transmitter vectorial workload in the bench's configuration:
    sampled transmitters' fields and masked data against the oracle."""
    cfg, f, tx, rx = synth.make_inputs("c7")
    build.build()
    ctx = cisor.Cisor(cfg["n"], cfg["delta"], tx, rx, dim=3, vectorial=True)
    ctx.set_rx_mask(cfg["rx_mask"])
    ctx.autotune()
    n, T = cfg["n"], cfg["T"]
    u = np.empty((T, 3, n, n, n), np.complex64)
    y = np.empty((T, ctx.M), np.complex64)
    st, info = ctx.forward(c64(f), u_out=u, y_out=y, tol=1e-4, max_iter=2000)
    assert info.n_not_converged == 0 and info.resid_max <= 1e-4
    ts = [0, 40, 80]
    prob = vector.VectorProblem(n, cfg["delta"], tx[ts, :3], tx[ts, 3:], rx, P=ctx.P)
    ref = vector.solve_fields(prob, f.astype(np.complex128), prob.u_in, tol=1e-10)
    for i, t in enumerate(ts):
        assert rel(u[t], ref[i]) < 2e-3   # GPU at residual 1e-4 vs FP64 at 1e-10
    assert rel(y[ts], prob.sense(f, ref)) < 2e-3
