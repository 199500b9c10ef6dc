"""Convergence of relaxed FISTA against its relaxation parameter alpha.

    python -m paper_1708_01663_gb300.alpha_sweep [--config c1] [--iters 40] [--alphas 0,0.5,0.8,0.96,1]

Sec. III-A's iteration (Eqs. 9-11) interpolates between ISTA (alpha = 0) and
FISTA (alpha = 1); the paper's analysis needs alpha < 1 and its experiments
use alpha = 0.96.  For each alpha this runs ``--iters`` steps of cisor_step
on a named synthetic workload (seeded phantom, measurements from the forward
model plus 40 dB noise), all from f_0 = 0 with the same step size, and prints
one JSON line per alpha: the data term D(s_k) of every iteration and the
reconstructed SNR 20 log10(||f_true|| / ||f_k - f_true||) (Sec. IV).

The step size is gamma = c / L, with L the largest eigenvalue of the
first-Born Hessian sum_t Re diag(u_in,t)^H H^H H diag(u_in,t), estimated by
power iteration through the library's sensing operators; c = ``--gamma-scale``.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np


def born_lipschitz(ctx, u_in, iters=30, seed=3):
    """Power iteration on x -> sum_t Re conj(u_in,t) H^H H (u_in,t x) (real x, [N])."""
    import torch
    dev = u_in.device
    T, N = u_in.shape
    g = torch.Generator(device="cpu").manual_seed(seed)
    x = torch.rand(N, generator=g, dtype=torch.float64).to(dev)
    Z = torch.empty((T, ctx.M), dtype=torch.complex64, device=dev)
    z = torch.empty((T, N), dtype=torch.complex64, device=dev)
    lam = 0.0
    for _ in range(iters):
        x = x / torch.linalg.vector_norm(x)
        xc = x.to(torch.complex64)
        ctx.sense(xc, u_in, Z)                   # Z_t = H (x u_in,t)
        ctx.sense_adjoint(xc, Z, z=z)            # z_t = H^H Z_t
        y = (torch.conj(u_in) * z).sum(0).real.to(torch.float64)
        lam = float(torch.dot(x, y))
        x = y
    return lam


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c1")
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--alphas", default="0,0.5,0.8,0.96,1")
    ap.add_argument("--gamma-scale", type=float, default=1.0)
    ap.add_argument("--tol", type=float, default=1e-5)
    args = ap.parse_args()
    import torch

    from paper_1708_01663_gb300 import build, cisor, synth
    build.build()
    dev = torch.device("cuda", 0)
    cfg, f_true, angles, rx = synth.make_inputs(args.config)
    n, T, M, dim = cfg["n"], cfg["T"], cfg["M"], cfg["dim"]
    complex_f = cfg["imag"] != 0.0
    ctx = cisor.Cisor(n, cfg["delta"], angles, rx, complex_f=complex_f, dim=dim, tx_kind=cfg.get("tx_kind", 0))
    if "rx_mask" in cfg:
        ctx.set_rx_mask(cfg["rx_mask"])
    f_dev = torch.from_numpy(np.ascontiguousarray(f_true, dtype=np.complex64)).to(dev)
    y = torch.empty((T, M), dtype=torch.complex64, device=dev)
    ctx.forward(f_dev, y_out=y, tol=1e-6, max_iter=5000, check=False)
    noise = torch.from_numpy(synth.complex_noise(cfg["seed"] + 100, (T, M)).astype(np.complex64)).to(dev)
    y += float(torch.linalg.vector_norm(y)) * 10 ** (-cfg["snr_db"] / 20) / math.sqrt(T * M) * noise
    u_in = torch.empty((T, ctx.N), dtype=torch.complex64, device=dev)
    ctx.incident(u_in)
    L = born_lipschitz(ctx, u_in)
    gamma = args.gamma_scale / L
    ft = f_true.astype(np.complex128)
    for a in (float(v) for v in args.alphas.split(",")):
        f = torch.zeros(f_dev.shape, dtype=torch.complex64, device=dev)
        s = torch.zeros_like(f)
        st = ctx.new_state(f, s, a, gamma, cfg["tau"], cfg["tv_iters"], 0.0, 2.0, 0.0, 0.5)
        Ds, snr = [], []
        for _ in range(args.iters):
            ctx.step(st, y, tol=args.tol, max_iter=5000, check=False)
            Ds.append(st.D)
            fk = f.cpu().numpy().astype(np.complex128)
            snr.append(20 * math.log10(np.linalg.norm(ft) / max(np.linalg.norm(fk - ft), 1e-300)))
        print(json.dumps({"config": args.config, "alpha": a, "gamma": gamma, "born_lipschitz": L,
                          "tau": cfg["tau"], "D": Ds, "snr_db": snr}), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
