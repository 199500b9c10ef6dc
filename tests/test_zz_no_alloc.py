"""The allocation-free matvec entry point against the context-based one.

cisor_apply_A_static serves callers that cannot call cudaMalloc (a host
framework that owns all device memory, or code that must not allocate while
a CUDA graph is captured).  It keeps its scratch in one file-scope device
array shared by every call.  Here it must reproduce cisor_apply_A on the same
inputs, within the matvec tolerance of the other parity tests, on two calls in
a row (the second call reuses the scratch the first left behind), and reject a
size beyond its scratch limit before touching the GPU.
"""
import numpy as np
import pytest

from paper_1708_01663_gb300 import build, cisor, synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(n, nvec):
    """A context of grid side n (FFT side P = 2n rounded up to a power of two, at least 64), its Green
    spectrum divided by P * P, and a seeded complex contrast, all on cuda:0."""
    import torch
    dev = torch.device("cuda", 0)
    ctx = cisor.Cisor(n, 1.0 / 8, synth.plane_wave_angles(nvec), synth.circle_receivers(8, n / 8.0 + 1.0))
    P = ctx.P
    ghat = torch.empty((P, P), dtype=torch.complex64, device=dev)
    ctx.green_spectrum(ghat)
    ghat_scaled = (ghat / (P * P)).contiguous()
    f = torch.from_numpy(synth.ellipse_phantom(n, 4, (0.0, 0.8), 21, 0.05).astype(np.complex64)).to(dev)
    return ctx, ghat_scaled, f


def _check_call(ctx, ghat_scaled, f, n, nvec, seed, adjoint):
    import torch
    x = torch.from_numpy(synth.random_field(seed, (nvec, n, n)).astype(np.complex64)).to(f.device)
    y_ref = torch.empty_like(x)
    ctx.apply_A(f, x, y_ref, adjoint=adjoint)
    y = torch.full_like(x, float("nan"))
    cisor.apply_A_static(ghat_scaled, f, x, y, n, ctx.P, adjoint=adjoint)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(y)).all()
    assert _rel(y.cpu().numpy(), y_ref.cpu().numpy()) < 2e-5


@pytest.mark.parametrize("n,nvec", [(32, 2), (64, 4), (128, 3), (256, 3)])
def test_static_matvec_matches_context_matvec(n, nvec):
    """P = 64, 128, 256 and 512; two calls in a row, the second reusing the scratch the first left."""
    build.build()
    ctx, ghat_scaled, f = _case(n, nvec)
    for call, adjoint in enumerate([False, True]):
        _check_call(ctx, ghat_scaled, f, n, nvec, 30 + call, adjoint)
    ctx.close()


def test_static_matvec_switches_fft_size():
    """Calls at P = 512, then 128, then 512 again: each call rewrites the shared stage-twiddle tables
    for its own FFT size before it reads them."""
    build.build()
    cases = {n: _case(n, 2) for n in (256, 64)}
    for i, n in enumerate((256, 64, 256)):
        ctx, ghat_scaled, f = cases[n]
        _check_call(ctx, ghat_scaled, f, n, 2, 40 + i, adjoint=bool(i % 2))
    for ctx, _, _ in cases.values():
        ctx.close()


def test_static_matvec_rejects_oversize():
    import torch
    build.build()
    n, P = 256, 512
    nvec = 17  # 8 * 17 * 256 * 512 bytes > 16 MiB scratch
    dev = torch.device("cuda", 0)
    g = torch.zeros((P, P), dtype=torch.complex64, device=dev)
    f = torch.zeros((n * n,), dtype=torch.complex64, device=dev)
    x = torch.zeros((nvec, n * n), dtype=torch.complex64, device=dev)
    with pytest.raises(cisor.CisorError) as err:
        cisor.apply_A_static(g, f, x, torch.empty_like(x), n, P)
    assert err.value.status == cisor.ERR_INVALID_ARG
    assert "maximum" in cisor.last_error()
