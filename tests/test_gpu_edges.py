"""Edge sizes of the CUDA path against the FP64 oracle: the smallest grids
(n = 8, FFT 64) with one transmitter and one receiver, the largest 3D grid
(n = 128, FFT 256^3) and the vectorial model at FFT 128^3 -- the kernel
instantiations the workload tests do not reach.  Bars as in the parity tests."""
import numpy as np
import pytest

from oracle import model, solve, vector
from paper_1708_01663_gb300 import build, cisor, synth
from tests.gpu_util import c64, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("adjoint", [False, True])
def test_smallest_2d_grid_one_transmitter_one_receiver(adjoint):
    build.build()
    n = 8
    angles, rx = np.array([0.3]), np.array([[2.0, 0.5]])
    ctx = cisor.Cisor(n, 1.0 / 8, angles, rx)
    assert (ctx.P, ctx.T, ctx.M) == (64, 1, 1)
    prob = model.Problem(n, 1.0 / 8, angles, rx, P=ctx.P)
    f = synth.disk_phantom(n, 1.0 / 8, 0.3, 0.8 + 0.05j)
    x = synth.random_field(3, (1, n, n))
    y = np.empty((1, n, n), np.complex64)
    ctx.apply_A(c64(f), c64(x), y, adjoint=adjoint)
    assert rel(y[0], (prob.AH if adjoint else prob.A)(f, x[0])) < 2e-5
    u = np.empty((1, n, n), np.complex64)
    yo = np.empty((1, 1), np.complex64)
    st, info = ctx.forward(c64(f), u_out=u, y_out=yo, tol=1e-6)
    ref, _, _ = solve.solve_fields(prob, f, prob.u_in, tol=1e-12)
    assert rel(u, ref) < 1e-4 and rel(yo, prob.sense(f, ref)) < 1e-4


def test_smallest_3d_grid():
    build.build()
    n = 8
    dirs = synth.hemisphere_directions()[:1]
    rx = np.array([[0.1, 0.2, 2.0]])
    ctx = cisor.Cisor(n, 1.0 / 6, dirs, rx, dim=3)
    assert ctx.P == 64
    prob = model.Problem(n, 1.0 / 6, dirs, rx, P=ctx.P, dim=3)
    f = synth.sphere_phantom(n, 2, (0.2, 0.6), 4, 0.02)
    u = np.empty((1, n, n, n), np.complex64)
    ctx.forward(c64(f), u_out=u, tol=1e-6)
    ref, _, _ = solve.solve_fields(prob, f, prob.u_in, tol=1e-12)
    assert rel(u, ref) < 1e-4


@pytest.mark.parametrize("adjoint", [False, True])
def test_largest_3d_grid(adjoint):
    """n = 128 (the 3D maximum): FFT side 256, the 3D column kernels at P = 256."""
    build.build()
    n = 128
    dirs = synth.hemisphere_directions()[:1]
    rx = np.array([[0.0, 0.0, 0.6 * n / 6 + 1.0]])
    ctx = cisor.Cisor(n, 1.0 / 6, dirs, rx, dim=3)
    assert ctx.P == 256
    k, kb = model.wavenumbers(1.0)
    ghat = model.green_spectrum(n, 256, 1.0 / 6, k, kb, dim=3)
    f = synth.sphere_phantom(n, 3, (0.1, 0.5), 9, 0.02)
    x = synth.random_field(10, (1, n, n, n))
    y = np.empty((1, n, n, n), np.complex64)
    ctx.apply_A(c64(f), c64(x), y, adjoint=adjoint)
    ref = (model.apply_AH if adjoint else model.apply_A)(f, x[0], ghat)
    assert rel(y[0], ref) < 2e-5


@pytest.mark.parametrize("adjoint", [False, True])
def test_vectorial_fft_128(adjoint):
    """The vectorial model at n = 40 (FFT 128 per component) and the smallest grid n = 8."""
    build.build()
    for n in (40, 8):
        tx = synth.polarised_hemisphere(2, 2)[:2]
        rx = np.array([[0.3, -0.2, 0.5 * n / 10 + 1.5]])
        ctx = cisor.Cisor(n, 0.1, tx, rx, dim=3, vectorial=True)
        assert ctx.P == (128 if n == 40 else 64)
        prob = vector.VectorProblem(n, 0.1, tx[:, :3], tx[:, 3:], rx, P=ctx.P)
        f = synth.sphere_phantom(n, 2, (0.2, 0.8), 6, 0.03)
        x = synth.random_field(12, (2, 3, n, n, n))
        y = np.empty((2, 3, n, n, n), np.complex64)
        ctx.apply_A(c64(f), c64(x), y, adjoint=adjoint)
        op = prob.AH if adjoint else prob.A
        for t in range(2):
            assert rel(y[t], op(f, x[t])) < 2e-5, (n, t)


def test_tensor_core_wait_gives_up_and_device_stays_usable():
    """The bounded wait every tensor-core kernel takes on its MMA barrier: completes when the barrier does,
    gives up after its poll limit when nothing completes it (no fault, no hang), and the device and a context
    keep working afterwards."""
    import time

    build.build()
    assert cisor.tc_wait_selftest(True, 1 << 20)
    t0 = time.time()
    assert not cisor.tc_wait_selftest(False, 2000)
    assert time.time() - t0 < 10.0
    assert cisor.tc_wait_selftest(True, 1 << 20)
    n, T, M = 16, 2, 4
    angles = synth.plane_wave_angles(T)
    rx = synth.circle_receivers(M, 3.0)
    ctx = cisor.Cisor(n, 1.0 / 8, angles, rx)
    prob = model.Problem(n, 1.0 / 8, angles, rx, P=ctx.P)
    f = synth.disk_phantom(n, 1.0 / 8, 0.5, 0.5 + 0.02j)
    u = synth.random_field(4, (T, n, n))
    Z = np.empty((T, M), np.complex64)
    ctx.sense(c64(f), c64(u), Z)
    assert rel(Z, prob.sense(f, u)) < 1e-5
