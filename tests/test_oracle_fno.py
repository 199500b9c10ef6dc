"""Pins of the FP64 FNO oracle: its hand-written backward against central finite
differences of the loss in every parameter group, and the spectral pair
against numpy's FFT (an independent library route)."""
import numpy as np
import pytest

from oracle import fno
from paper_1708_01663_gb300 import synth


def _small():
    n, C, m, L, H = 16, 4, 3, 3, 6
    p = fno.init_params(n, C, m, L, H, seed=3)
    for k in p:
        if k.startswith("b") or k.startswith("c"):
            p[k] = 0.1 * synth.random_field(hash(k) % 1000, p[k].shape).real
    fs = [synth.ellipse_phantom(n, 2, (0.1, 0.5), 5 + b, 0.02) for b in range(2)]
    u = [np.exp(1j * (0.7 * b + np.add.outer(np.arange(n), 0.5 * np.arange(n)) * 0.4)) for b in range(2)]
    t = [synth.random_field(20 + b, (n, n)) for b in range(2)]
    return p, fs, u, t, L


def test_analysis_matches_numpy_fft():
    n, m = 16, 3
    v = synth.random_field(1, (n, n)).real
    Fx, Fy, w = fno.dft_mats(n, m)
    X = fno.analysis(v, Fx, Fy)
    full = np.fft.fft2(v)
    ref = full[np.ix_(fno.kx_modes(n, m), np.arange(m))]
    assert np.abs(X - ref).max() < 1e-12


def test_synthesis_is_irfft2_of_truncated_spectrum():
    # with every mode kept (m = n/2 plus the Nyquist-free half), Lsyn inverts S on band-limited real images
    n, m = 16, 4
    Fx, Fy, w = fno.dft_mats(n, m)
    spec = np.zeros((n, n // 2 + 1), complex)
    rng = synth.random_field(2, (2 * m, m))
    rng[:, 0] = 0  # ky = 0 column handled by Re
    spec[np.ix_(fno.kx_modes(n, m), np.arange(m))] = rng
    img = np.fft.irfft2(spec, s=(n, n))
    back = fno.synthesis(fno.analysis(img, Fx, Fy), Fx, Fy, w, 1.0 / (n * n))
    assert np.abs(back - img).max() < 1e-12


@pytest.mark.parametrize("group", ["W0", "b0", "R0", "R2", "W1", "W3", "b2", "P1", "c1", "P2", "c2"])
def test_backward_matches_central_differences(group):
    p, fs, u, t, L = _small()
    val, g = fno.loss_and_grad(p, fs, u, t, L)
    assert abs(val - fno.loss(p, fs, u, t, L)) < 1e-12
    idx = [tuple(i) for i in np.argwhere(np.ones(p[group].shape))[:: max(1, p[group].size // 5)][:5]]
    h = 1e-6
    for ix in idx:
        for unit in ([1.0, 1j] if np.iscomplexobj(p[group]) else [1.0]):
            pp = {k: v.copy() for k, v in p.items()}
            pm = {k: v.copy() for k, v in p.items()}
            pp[group][ix] += h * unit
            pm[group][ix] -= h * unit
            fd = (fno.loss(pp, fs, u, t, L) - fno.loss(pm, fs, u, t, L)) / (2 * h)
            an = g[group][ix].real if unit == 1.0 else g[group][ix].imag
            assert abs(fd - an) < 1e-6 * max(1.0, abs(fd)), (group, ix, unit, fd, an)
