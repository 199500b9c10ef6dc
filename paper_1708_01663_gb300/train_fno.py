"""Train the learned warm start on solver-generated fields and measure its gain.

    python -m paper_1708_01663_gb300.train_fno [--train 2000] [--test 200] [--minutes 3] [--save FILE]

Workload: 128 x 128 grids at lambda/8 (FFT 256 x 256), 32 plane-wave
transmitters, phantoms of 3-10 seeded random ellipses with real contrast in
[0, 0.8].  Targets are the demodulated scattered fields conj(u_in)(u - u_in)
of the solver's own forward solves (tolerance 1e-6); the warm start is
u_in (1 + network).  Training: Adam on batches of 32 random
(phantom, transmitter) samples, learning rate 1e-3 decayed by cosine over the
time budget.  Evaluation on held-out phantoms: cold-start solves (x0 = u_in)
against warm-started solves (x0 = u_in + network), both to relative residual
1e-4, timed with CUDA events (the warm time includes the network inference).
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

N, T, DELTA = 128, 32, 1.0 / 8


def phantom(i, seed0=1712000):
    from paper_1708_01663_gb300 import synth
    count = 3 + int(synth.Rng(seed0 + 7 * i).uniform(0, 8, 1)[0])
    return synth.ellipse_phantom(N, count, (0.0, 0.8), seed0 + i)


def geometry():
    from paper_1708_01663_gb300 import synth
    return synth.plane_wave_angles(T), synth.circle_receivers(64, 12.0)


def generate(ctx, idx, dev, tol=1e-6):
    """Phantoms and the scattered fields of all T transmitters, on the device."""
    import torch
    fs = torch.empty((len(idx), N * N), dtype=torch.complex64, device=dev)
    us = torch.empty((len(idx), T, N * N), dtype=torch.complex64, device=dev)
    u_in = torch.empty((T, N * N), dtype=torch.complex64, device=dev)
    ctx.incident(u_in)
    u = torch.empty((T, N * N), dtype=torch.complex64, device=dev)
    for k, i in enumerate(idx):
        fs[k] = torch.from_numpy(phantom(i).astype(np.complex64).ravel()).to(dev)
        ctx.forward(fs[k], u_out=u, tol=tol, max_iter=5000, check=False)
        us[k] = (u - u_in) * torch.conj(u_in)  # demodulated scattered field (|u_in| = 1)
    return fs, us, u_in


def train(net, fs, usc, u_in, minutes, lr0=1e-3, B=32, seed=5):
    import torch
    dev = fs.device
    P = fs.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    t_end = time.time() + 60.0 * minutes
    steps, losses = 0, []
    t0 = time.time()
    while time.time() < t_end:
        frac = min(1.0, (time.time() - t0) / (60.0 * minutes))
        lr = lr0 * 0.5 * (1.0 + math.cos(math.pi * frac)) + 1e-5
        pi = torch.randint(0, P, (B,), generator=g).to(dev)
        ti = torch.randint(0, T, (B,), generator=g).to(dev)
        f = fs[pi].contiguous()
        ui = u_in[ti].contiguous()
        tg = usc[pi, ti].contiguous()
        losses.append(net.train_step(f, ui, tg, lr))
        steps += 1
    return steps, losses


def evaluate(ctx, net, idx, dev, tol=1e-4):
    import torch
    res = {"cold_iters": [], "warm_iters": [], "cold_ms": [], "warm_ms": [], "pred_err": [], "infer_ms": []}
    u_in = torch.empty((T, N * N), dtype=torch.complex64, device=dev)
    ctx.incident(u_in)
    u = torch.empty((T, N * N), dtype=torch.complex64, device=dev)
    x0 = torch.empty_like(u)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    for i in idx:
        f = torch.from_numpy(phantom(i).astype(np.complex64).ravel()).to(dev)
        torch.cuda.synchronize()
        ev[0].record()
        _, ic = ctx.forward(f, u_out=u, tol=tol, max_iter=5000, x0_mode=0, check=False)
        ev[1].record()
        u_ref = u.clone()
        ev[2].record()
        net.warm_start(ctx, f, x0)
        ev[4].record()
        _, iw = ctx.forward(f, x0=x0, u_out=u, tol=tol, max_iter=5000, x0_mode=1, check=False)
        ev[3].record()
        torch.cuda.synchronize()
        res["infer_ms"].append(ev[2].elapsed_time(ev[4]))
        res["cold_iters"].append(ic.iters_mean)
        res["warm_iters"].append(iw.iters_mean)
        res["cold_ms"].append(ev[0].elapsed_time(ev[1]))
        res["warm_ms"].append(ev[2].elapsed_time(ev[3]))
        sc_true = u_ref - u_in
        res["pred_err"].append(float(torch.linalg.vector_norm(x0 - u_ref) / torch.linalg.vector_norm(sc_true)))
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--minutes", type=float, default=3.0)
    ap.add_argument("--save", default=None)
    args = ap.parse_args()
    import torch

    from paper_1708_01663_gb300 import build, cisor
    build.build()
    dev = torch.device("cuda", 0)
    ang, rx = geometry()
    ctx = cisor.Cisor(N, DELTA, ang, rx)
    t0 = time.time()
    fs, usc, u_in = generate(ctx, range(args.train), dev)
    t_gen = time.time() - t0
    net = cisor.FNO(max_batch=T, seed=1714)
    t0 = time.time()
    steps, losses = train(net, fs, usc, u_in, args.minutes)
    t_train = time.time() - t0
    del fs, usc
    test_idx = range(100000, 100000 + args.test)
    ev = evaluate(ctx, net, test_idx, dev)
    if args.save:
        flat = np.empty(net.num_params, np.float32)
        net.get_params(flat, as_used=False)
        flat.tofile(args.save)
    ci, wi = np.mean(ev["cold_iters"]), np.mean(ev["warm_iters"])
    cm, wm = np.mean(ev["cold_ms"]), np.mean(ev["warm_ms"])
    print(json.dumps({
        "workload": "128x128 at lambda/8 (FFT 256), 32 Tx, 3-10 ellipses contrast [0, 0.8]; residual 1e-4",
        "train_phantoms": args.train, "test_phantoms": args.test, "samples": args.train * T,
        "gen_s": t_gen, "train_s": t_train, "steps": steps, "batch": 32,
        "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-50:])),
        "pred_rel_err_mean": float(np.mean(ev["pred_err"])),
        "cold_iters_mean": ci, "warm_iters_mean": wi, "iters_saved_frac": 1.0 - wi / ci,
        "cold_ms_mean": cm, "warm_ms_mean": wm, "time_saved_frac": 1.0 - wm / cm,
        "infer_ms_mean": float(np.mean(ev["infer_ms"])),
        "cold_solves_per_s": T / (cm / 1e3), "learned_solves_per_s": T / (wm / 1e3),
        "warm_iters_p95": float(np.percentile(ev["warm_iters"], 95)),
        "cold_iters_p95": float(np.percentile(ev["cold_iters"], 95))}))
    net.close()
    ctx.close()


if __name__ == "__main__":
    main()
