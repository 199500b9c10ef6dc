"""torch.autograd.Function over the CUDA data term: the backward (adjoint solve)
against central finite differences of the FP64 oracle's D (step 1e-3 on 16
seeded pixels), against the oracle gradient, and against finite differences of
the GPU's own D."""
import numpy as np
import pytest

from oracle import grad as ograd
from paper_1708_01663_gb300 import synth
from tests.gpu_util import c64, make, rel

pytestmark = pytest.mark.gpu


def _setup(complex_f):
    import torch
    n, T, M = 48, 4, 24
    ctx, prob = make(n, T, M, 5.0, complex_f=complex_f)
    imag = 0.03 if complex_f else 0.0
    f = synth.ellipse_phantom(n, 3, (0.1, 0.5), 12, imag)
    f_true = synth.ellipse_phantom(n, 3, (0.1, 0.6), 13, imag)
    _, y, _, _ = ograd.forward(prob, f_true, tol=1e-12)
    return torch, ctx, prob, f, y


@pytest.mark.parametrize("complex_f", [False, True])
def test_autograd_matches_oracle_and_fd(complex_f):
    torch, ctx, prob, f, y = _setup(complex_f)
    from paper_1708_01663_gb300.autograd import data_term
    dev = torch.device("cuda", 0)
    ft = torch.from_numpy(c64(f) if complex_f else np.ascontiguousarray(f.real, np.float32)).to(dev)
    ft.requires_grad_(True)
    yt = torch.from_numpy(c64(y)).to(dev)
    D = data_term(ft, yt, ctx, tol=1e-7)
    D.backward()
    g = ft.grad.detach().cpu().numpy()
    D_ref, g_ref = ograd.data_and_grad(prob, f, y, tol=1e-12)
    assert abs(D.item() - D_ref) / D_ref < 1e-4
    gref = g_ref if complex_f else g_ref.real
    assert rel(g, gref) < 5e-4
    # central differences of the FP64 oracle's D, step 1e-3, 16 seeded pixels
    rng = synth.Rng(99)
    pix = (rng.uniform(0, 1, 16) * f.size).astype(int)
    h = 1e-3
    scale = np.abs(gref).max()
    for p in pix:
        iy, ix = divmod(int(p), f.shape[1])
        for unit in ([1.0, 1j] if complex_f else [1.0]):
            fp = f.copy(); fp[iy, ix] += h * unit
            fm = f.copy(); fm[iy, ix] -= h * unit
            fd = (ograd.data_term(prob, fp, y, 1e-12) - ograd.data_term(prob, fm, y, 1e-12)) / (2 * h)
            an = g[iy, ix].real if unit == 1.0 else g[iy, ix].imag
            assert abs(fd - an) < 2e-3 * scale, (iy, ix, unit, fd, an)


def test_autograd_gpu_finite_differences():
    torch, ctx, prob, f, y = _setup(False)
    from paper_1708_01663_gb300.autograd import data_term
    dev = torch.device("cuda", 0)
    ft = torch.from_numpy(np.ascontiguousarray(f.real, np.float32)).to(dev).requires_grad_(True)
    yt = torch.from_numpy(c64(y)).to(dev)
    D = data_term(ft, yt, ctx, tol=1e-7)
    D.backward()
    g = ft.grad.detach().cpu().numpy()
    rng = synth.Rng(7)
    pix = (rng.uniform(0, 1, 16) * f.size).astype(int)
    h = 1e-3
    scale = np.abs(g).max()
    with torch.no_grad():
        for p in pix:
            e = torch.zeros_like(ft).view(-1)
            e[int(p)] = h
            e = e.view_as(ft)
            dp = data_term(ft + e, yt, ctx, tol=1e-7).item()
            dm = data_term(ft - e, yt, ctx, tol=1e-7).item()
            fd = (dp - dm) / (2 * h)
            assert abs(fd - g.reshape(-1)[int(p)]) < 3e-2 * scale


def test_backward_survives_calls_that_only_read_f():
    """cisor_data_backward differentiates at the point of the last cisor_data_term (Prop. 1) even when
    calls that overwrite the context's f come in between; calls that overwrite the kept u or w make it
    refuse instead of differentiating at another point."""
    _, ctx, prob, f, y = _setup(False)
    from paper_1708_01663_gb300 import cisor
    fc = c64(f)
    D, _, _ = ctx.data_term(fc, c64(y), tol=1e-7)
    other = c64(synth.ellipse_phantom(prob.n, 2, (0.0, 0.9), 77))
    x = c64(synth.random_field(5, (ctx.T, prob.n, prob.n)))
    out = np.empty_like(x)
    ctx.apply_A(other, x, out)
    ctx.autotune(reps=1)
    ctx.tv_prox(other, np.empty_like(other), 1e-3, 5)
    g = np.empty(fc.shape, np.complex64)
    ctx.data_backward(g, tol=1e-7)
    D_ref, g_ref = ograd.data_and_grad(prob, f, y, tol=1e-12)
    assert abs(D - D_ref) / D_ref < 1e-4
    assert rel(g.real, g_ref.real) < 5e-4
    # a forward solve overwrites the kept fields: the backward is refused
    ctx.data_term(fc, c64(y), tol=1e-7)
    ctx.forward(other, tol=1e-5)
    with pytest.raises(cisor.CisorError) as ei:
        ctx.data_backward(g, tol=1e-7)
    assert ei.value.status == cisor.ERR_INVALID_ARG
