"""Fresnel-style geometry on the CUDA path vs the FP64 oracle (Sec. IV set-ups):
point / line-source transmitters, per-transmitter receiver masks, and several
frequencies reconstructed together (one context per frequency, gradients
summed before cisor_step_update).  Bars as in the other parity tests."""
import numpy as np
import pytest

from oracle import fista, grad, model
from paper_1708_01663_gb300 import build, cisor, synth
from tests.gpu_util import c64, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ctx(n, delta, src, rx, dim=2, complex_f=False, wavelength=1.0):
    build.build()
    ctx = cisor.Cisor(n, delta, src, rx, dim=dim, tx_kind="point", complex_f=complex_f, wavelength=wavelength)
    prob = model.Problem(n, delta, src, rx, P=ctx.P, dim=dim, tx_kind="point", wavelength=wavelength)
    return ctx, prob


@pytest.mark.parametrize("dim", [2, 3])
def test_point_source_tables(dim):
    n = 40 if dim == 2 else 16
    delta = 1.0 / 8 if dim == 2 else 1.0 / 6
    if dim == 2:
        src, rx = synth.circle_sources(5, 4.0, 0.3), synth.circle_receivers(24, 4.5)
    else:
        src = np.array([[2.5, 0.1, 0.3], [-0.2, 2.4, -0.5], [0.3, 0.4, -2.6]])
        rx = synth.planar_receivers(4, 0.5, 2.0)
    ctx, prob = _ctx(n, delta, src, rx, dim=dim)
    u = np.empty((ctx.T,) + (n,) * dim, np.complex64)
    ctx.incident(u)
    assert rel(u, prob.u_in) < 1e-6


def test_point_source_inside_grid_rejected():
    build.build()
    with pytest.raises(cisor.CisorError):
        cisor.Cisor(40, 1.0 / 8, np.array([[0.5, 0.2]]), synth.circle_receivers(8, 4.0), tx_kind="point")


@pytest.mark.parametrize("complex_f", [False, True])
def test_masked_gradient(complex_f):
    n, T, M = 48, 6, 40
    src, rx = synth.circle_sources(T, 4.5), synth.circle_receivers(M, 5.0)
    mask = synth.angular_mask(src, rx, 60.0)
    ctx, prob = _ctx(n, 1.0 / 8, src, rx, complex_f=complex_f)
    imag = 0.03 if complex_f else 0.0
    f = synth.ellipse_phantom(n, 3, (0.1, 0.5), 12, imag)
    f_true = synth.ellipse_phantom(n, 3, (0.1, 0.6), 13, imag)
    _, y, _, _ = grad.forward(prob, f_true, tol=1e-12)
    y = y + 50.0 * (1 - mask) * synth.random_field(5, y.shape)   # junk at inactive receivers must not matter
    D_ref, g_ref = grad.data_and_grad(prob, f, y, tol=1e-12, mask=mask)
    ctx.set_rx_mask(mask)
    g = np.empty((n, n), np.complex64)
    D, st, info = ctx.grad(c64(f), c64(y), g, tol=1e-6, max_iter=3000)
    assert abs(D - D_ref) / D_ref < 1e-4
    assert rel(g if complex_f else g.real, g_ref if complex_f else g_ref.real) < 5e-4
    # clearing the mask brings the junk back into D
    ctx.set_rx_mask(None)
    D_all, _, _ = ctx.grad(c64(f), c64(y), g, tol=1e-6, max_iter=3000)
    assert D_all > 100 * D


def test_two_frequency_reconstruction_steps():
    n, T, M = 48, 6, 36
    src, rx = synth.circle_sources(T, 4.5), synth.circle_receivers(M, 5.0)
    mask = synth.angular_mask(src, rx, 60.0)
    waves = [1.0, 0.8]
    ctxs, probs = zip(*[_ctx(n, 1.0 / 8, src, rx, wavelength=w) for w in waves])
    f_true = synth.ellipse_phantom(n, 3, (0.0, 0.4), 21)
    ys = [grad.forward(p, f_true, tol=1e-12)[1] for p in probs]
    for ctx in ctxs:
        ctx.set_rx_mask(mask)
    s0 = np.zeros((n, n))
    # step size from the oracle gradient scale at f = 0 (an input on both sides)
    g0 = sum(grad.data_and_grad(p, s0, y, tol=1e-12, mask=mask)[1] for p, y in zip(probs, ys))
    gamma = 0.2 * float(np.linalg.norm(f_true)) / float(np.linalg.norm(g0.real))
    tau, alpha, K, tv_iters = 1e-3, 0.96, 4, 10

    def both(s, state):
        Ds, gs = zip(*[grad.data_and_grad(p, s, y, tol=1e-12, mask=mask) for p, y in zip(probs, ys)])
        return sum(Ds), sum(gs)

    ref, hist = fista.relaxed_fista(probs[0], None, s0, gamma, tau, alpha, K, tv_iters, grad_fn=both)
    dev = torch.device("cuda")
    ys_d = [torch.from_numpy(c64(y)).to(dev) for y in ys]
    bufs = [(torch.zeros((n, n), dtype=torch.complex64, device=dev),
             torch.zeros((n, n), dtype=torch.complex64, device=dev)) for _ in ctxs]
    states = [c.new_state(f, s, alpha, gamma, tau, tv_iters, 0.0, 2.0) for c, (f, s) in zip(ctxs, bufs)]
    g = [torch.empty((n, n), dtype=torch.complex64, device=dev) for _ in ctxs]
    Ds = []
    for _ in range(K):
        parts = [c.grad(s, y, gi, tol=1e-6, max_iter=3000, x0_mode=2)[0]
                 for c, (f, s), y, gi in zip(ctxs, bufs, ys_d, g)]
        gsum = g[0] + g[1]
        for c, st, gi in zip(ctxs, states, g):
            gi.copy_(gsum)
            c.step_update(st, gi, sum(parts))
        Ds.append(sum(parts))
    torch.cuda.synchronize()
    assert torch.equal(bufs[0][0], bufs[1][0])
    assert rel(Ds, hist) < 1e-3
    assert rel(bufs[0][0].cpu().numpy(), ref) < 1e-3


def test_c6_full_size_sampled():
    """The Fresnel-style workload at full size: masked forward data of sampled
    transmitters against the oracle."""
    cfg, f, src, rx = synth.make_inputs("c6")
    ctx, prob = _ctx(cfg["n"], cfg["delta"], src[[0, 5]], rx)
    assert ctx.P == 256
    u = np.empty((2, cfg["n"], cfg["n"]), np.complex64)
    y = np.empty((2, cfg["M"]), np.complex64)
    st, info = ctx.forward(c64(f), u_out=u, y_out=y, tol=1e-6, max_iter=3000)
    from oracle import solve
    ref, _, _ = solve.solve_fields(prob, f, prob.u_in, tol=1e-12)
    assert rel(u, ref) < 1e-4
    assert rel(y, prob.sense(f, ref)) < 1e-4
