"""FP64 Fourier neural operator (FNO) for the learned warm start -- TEST INFRASTRUCTURE.

Not from the paper: the learned initial guess of the field solves that the
GPU build adds on top of CISOR.  This module is the plain restatement of the
network the CUDA kernels implement, with a hand-written backward pass, used
to check the GPU forward values and parameter gradients.

Network for one sample (grid n x n, width C, m modes, L layers, hidden H):
  features   a = (Re f, Im f, Re u_in, Im u_in, d_x, d_y, x, y)  8 x n x n
             d = local propagation direction of u_in: the unit vector along
             (Im(conj u g_x), Im(conj u g_y)), g = central differences with
             clamped edges (0 where that vector vanishes)
  lifting    v0 = W0 a + b0                                       C x n x n (1x1 conv)
  layer l    X  = S(v_{l-1})      truncated DFT, per channel      C x 2m x m complex
             Y[o] = sum_i R_l[:, :, i, o] X[i]                    per mode
             pre = Lsyn(Y) + W_l v_{l-1} + b_l
             v_l = GELU(pre)  (no GELU after the last layer)
  projection z = P1 v_L + c1, h = GELU(z), out = P2 h + c2         2 x n x n
  output     e = out[0] + j out[1]; the warm start predicts u_sc = u_in * e
             (targets are the demodulated fields conj(u_in) u_sc)
S keeps the frequencies kx in {0..m-1, n-m..n-1} along rows (iy) and
ky in {0..m-1} along columns (ix):
  S(v)[kx, ky] = sum_{iy, ix} v[iy, ix] exp(-2 pi j (kx iy + ky ix) / n),
and the synthesis is the real part of the truncated inverse with the
negative-ky half folded in (weight 2 for ky > 0):
  Lsyn(Y)[iy, ix] = (1/n^2) Re sum_{kx, ky} w_ky Y[kx, ky] exp(+2 pi j (kx iy + ky ix) / n).
GELU(x) = x (1 + erf(x / sqrt 2)) / 2.  Loss = mean over samples of
||out - t|| / ||t|| (relative L2 of the scattered field).

Gradients of complex parameters are returned as dL/dRe + j dL/dIm.
Pinned by: central finite differences of the loss in every parameter group
(tests/test_oracle_fno.py).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def kx_modes(n, m):
    return np.r_[0:m, n - m:n]


def dft_mats(n, m):
    iy = np.arange(n)
    Fx = np.exp(-2j * np.pi * np.outer(kx_modes(n, m), iy) / n)        # [2m, n]
    Fy = np.exp(-2j * np.pi * np.outer(np.arange(m), iy) / n)          # [m, n]
    w = np.where(np.arange(m) == 0, 1.0, 2.0)
    return Fx, Fy, w


def analysis(v, Fx, Fy):
    """S(v) for v [..., n, n] -> [..., 2m, m]."""
    return Fx @ v @ Fy.T


def synthesis(Y, Fx, Fy, w, scale):
    """scale * Re sum_{kx,ky} w_ky Y exp(+...) for Y [..., 2m, m] -> [..., n, n]."""
    return scale * np.real(np.conj(Fx).T @ (Y * w) @ np.conj(Fy))


def _es(sub, *ops):
    return np.einsum(sub, *ops, optimize=True)


def gelu(x):
    return 0.5 * x * (1.0 + special.erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + special.erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def direction(u):
    """Unit local propagation direction of a field from its phase gradient."""
    up = np.pad(u, 1, mode="edge")
    gx = (up[1:-1, 2:] - up[1:-1, :-2]) / 2.0
    gy = (up[2:, 1:-1] - up[:-2, 1:-1]) / 2.0
    vx = np.imag(np.conj(u) * gx)
    vy = np.imag(np.conj(u) * gy)
    nv = np.sqrt(vx * vx + vy * vy)
    safe = np.where(nv > 0, nv, 1.0)
    return np.where(nv > 0, vx / safe, 0.0), np.where(nv > 0, vy / safe, 0.0)


def features(f, u_in, n):
    c = (np.arange(n) + 0.5) / n - 0.5
    Y, X = np.meshgrid(c, c, indexing="ij")
    dx, dy = direction(u_in)
    return np.stack([f.real, f.imag, u_in.real, u_in.imag, dx, dy, X, Y])


def init_params(n=128, C=32, m=16, L=4, H=128, seed=0):
    """Seeded initial parameters (same recipe as the CUDA initialiser is NOT required:
    tests pass the GPU's parameters in)."""
    rng = np.random.default_rng(seed)
    p = {"W0": rng.uniform(-1, 1, (C, 8)) / math.sqrt(8), "b0": np.zeros(C)}
    for l in range(L):
        p[f"R{l}"] = (rng.uniform(-1, 1, (2 * m, m, C, C)) + 1j * rng.uniform(-1, 1, (2 * m, m, C, C))) / C
        p[f"W{l + 1}"] = rng.uniform(-1, 1, (C, C)) / math.sqrt(C)
        p[f"b{l + 1}"] = np.zeros(C)
    p["P1"] = rng.uniform(-1, 1, (H, C)) / math.sqrt(C)
    p["c1"] = np.zeros(H)
    p["P2"] = rng.uniform(-1, 1, (2, H)) / math.sqrt(H)
    p["c2"] = np.zeros(2)
    return p


def forward(p, f, u_in, L=4):
    """u_sc prediction for one sample and the cache for backward."""
    n = f.shape[0]
    m = p["R0"].shape[1]
    Fx, Fy, w = dft_mats(n, m)
    a = features(f, u_in, n)
    v = _es("oc,cyx->oyx", p["W0"], a) + p["b0"][:, None, None]
    cache = {"a": a, "v": [v], "X": [], "pre": []}
    for l in range(L):
        X = analysis(v, Fx, Fy)                                      # [C, 2m, m]
        Ym = _es("klio,ikl->okl", p[f"R{l}"], X)               # [C, 2m, m]
        s = synthesis(Ym, Fx, Fy, w, 1.0 / (n * n))
        pre = s + _es("oi,iyx->oyx", p[f"W{l + 1}"], v) + p[f"b{l + 1}"][:, None, None]
        cache["X"].append(X)
        cache["pre"].append(pre)
        v = gelu(pre) if l < L - 1 else pre
        cache["v"].append(v)
    z = _es("hc,cyx->hyx", p["P1"], v) + p["c1"][:, None, None]
    h = gelu(z)
    out = _es("oh,hyx->oyx", p["P2"], h) + p["c2"][:, None, None]
    cache.update(z=z, h=h)
    return out[0] + 1j * out[1], cache


def loss_and_grad(p, fs, u_ins, targets, L=4):
    """Mean relative L2 loss over samples and its gradient in every parameter."""
    B = len(fs)
    g = {k: np.zeros_like(v) for k, v in p.items()}
    total = 0.0
    for b in range(B):
        pred, cache = forward(p, fs[b], u_ins[b], L)
        n = fs[b].shape[0]
        m = p["R0"].shape[1]
        Fx, Fy, w = dft_mats(n, m)
        diff = pred - targets[b]
        nd, nt = np.linalg.norm(diff), np.linalg.norm(targets[b])
        total += nd / nt
        dpred = diff / (nd * nt * B)                                  # d loss / d(Re) + j d / d(Im)
        dout = np.stack([dpred.real, dpred.imag])                     # [2, n, n]
        g["P2"] += _es("oyx,hyx->oh", dout, cache["h"])
        g["c2"] += dout.sum(axis=(1, 2))
        dh = _es("oh,oyx->hyx", p["P2"], dout)
        dz = dh * gelu_grad(cache["z"])
        vL = cache["v"][L]
        g["P1"] += _es("hyx,cyx->hc", dz, vL)
        g["c1"] += dz.sum(axis=(1, 2))
        dv = _es("hc,hyx->cyx", p["P1"], dz)
        for l in range(L - 1, -1, -1):
            pre = cache["pre"][l]
            dpre = dv * gelu_grad(pre) if l < L - 1 else dv
            vprev = cache["v"][l]
            g[f"W{l + 1}"] += _es("oyx,iyx->oi", dpre, vprev)
            g[f"b{l + 1}"] += dpre.sum(axis=(1, 2))
            dv = _es("oi,oyx->iyx", p[f"W{l + 1}"], dpre)
            dY = analysis(dpre, Fx, Fy) * w / (n * n)                 # adjoint of the synthesis
            X = cache["X"][l]
            g[f"R{l}"] += _es("ikl,okl->klio", np.conj(X), dY)
            dX = _es("klio,okl->ikl", np.conj(p[f"R{l}"]), dY)
            dv += synthesis(dX, Fx, Fy, np.ones_like(w), 1.0)          # adjoint of the analysis
        g["W0"] += _es("oyx,cyx->oc", dv, cache["a"])
        g["b0"] += dv.sum(axis=(1, 2))
    return total / B, g


def loss(p, fs, u_ins, targets, L=4):
    tot = 0.0
    for b in range(len(fs)):
        pred, _ = forward(p, fs[b], u_ins[b], L)
        tot += np.linalg.norm(pred - targets[b]) / np.linalg.norm(targets[b])
    return tot / len(fs)
