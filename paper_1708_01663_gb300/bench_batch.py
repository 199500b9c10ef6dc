"""Throughput of uneven problems solved together vs one after another.

    python -m paper_1708_01663_gb300.bench_batch [--reps 3]

Workload: four 2D problems with grids 96, 128, 192 and 256 at lambda/8 (FFT
sides 256, 256, 512, 512), 32 / 64 / 96 / 128 plane-wave transmitters
(assigned to the grids by a seeded shuffle), 128 receivers on a circle at 1.5
half-widths, seeded random ellipses with contrast in [0, 0.8] plus 0.02i.
Cold-start forward solves to relative residual 1e-4.  Prints one JSON line:
LS field solves per second for the batch (one CUDA-graph launch per solve: a
device-side WHILE loop over chunks of iterations advancing every problem) and
for the same contexts solved sequentially, both timed with CUDA events on the
caller's stream; and both again with the host-driven chunk loop.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

GRIDS = (96, 128, 192, 256)
TXS = (32, 64, 96, 128)


def workload(seed=1713):
    from paper_1708_01663_gb300 import synth
    order = np.argsort(synth.Rng(seed).uniform(count=len(TXS)))
    geoms, fs = [], []
    for i, n in enumerate(GRIDS):
        T = TXS[order[i]]
        geoms.append(dict(n=n, delta=1.0 / 8, tx_angles=synth.plane_wave_angles(T),
                          rx_pos=synth.circle_receivers(128, 1.5 * n / 16.0), complex_f=True))
        fs.append(synth.ellipse_phantom(n, 6, (0.0, 0.8), seed + 10 * i, 0.02).astype(np.complex64))
    return geoms, fs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tol", type=float, default=1e-4)
    args = ap.parse_args()
    import torch

    from paper_1708_01663_gb300 import build, cisor
    build.build()
    dev = torch.device("cuda", 0)
    geoms, fs = workload()
    fd = [torch.from_numpy(f).to(dev) for f in fs]
    batch = cisor.Batch(geoms, autotune=True)
    solves = sum(len(g["tx_angles"]) for g in geoms)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.reps

    infos = {}

    def run_batch():
        _, inf = batch.forward(fd, tol=args.tol, max_iter=5000, check=False)
        infos["batch"] = [i.as_dict() for i in inf]

    def run_seq():
        out = []
        for p, f in zip(batch.problems, fd):
            _, inf = p.forward(f, tol=args.tol, max_iter=5000, check=False)
            out.append(inf.as_dict())
        infos["seq"] = out

    ms_batch = timed(run_batch)
    ms_seq = timed(run_seq)
    batch.set_solve_loop(False)  # the host-driven chunk loop, for comparison
    for p in batch.problems:
        p.set_solve_loop(False)
    ms_batch_host = timed(run_batch)
    ms_seq_host = timed(run_seq)
    batch.set_solve_loop(True)
    for p in batch.problems:
        p.set_solve_loop(True)
    print(json.dumps({
        "workload": "grids 96/128/192/256, 32-128 Tx each, 128 Rx, contrast<=0.8+0.02i, cold start to 1e-4",
        "solves": solves, "batch_ms": ms_batch, "sequential_ms": ms_seq,
        "batch_solves_per_s": solves / (ms_batch / 1e3), "sequential_solves_per_s": solves / (ms_seq / 1e3),
        "speedup": ms_seq / ms_batch,
        "host_loop": {"batch_ms": ms_batch_host, "sequential_ms": ms_seq_host,
                      "what": "the same solves with the host replaying a 4-iteration chunk graph and reading the "
                              "active flags after every chunk"},
        "tuning": [p.tuning() for p in batch.problems],
        "P": [p.P for p in batch.problems], "T": [p.T for p in batch.problems],
        "iters_max": [i["iters_max"] for i in infos["batch"]],
        "iters_mean": [round(i["iters_mean"], 1) for i in infos["batch"]],
        "resid_max": max(i["resid_max"] for i in infos["batch"])}))
    batch.close()


if __name__ == "__main__":
    main()
