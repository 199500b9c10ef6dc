"""Time the FNO's inference and training step (and give a profiler something to capture).

    python -m paper_1708_01663_gb300.profile_fno [--batch 32] [--reps 10]

Builds a network for 128 x 128 grids, seeded phantoms, a random incident
field and random targets of the workload's shapes, runs 3 untimed and
``reps`` timed inferences, then 2 untimed and ``reps`` timed Adam steps, and
prints the milliseconds of each with CUDA events.  A launch list of the
same command:
``ncu --metrics gpu__time_duration.sum --clock-control none -k regex:fno_ -c 500``.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--reps", type=int, default=10)
    args = ap.parse_args()
    import torch

    from paper_1708_01663_gb300 import build, cisor, synth
    build.build()
    dev = torch.device("cuda", 0)
    B = args.batch
    net = cisor.FNO(max_batch=B, seed=3)
    f = torch.from_numpy(np.stack([synth.ellipse_phantom(128, 4, (0.0, 0.8), i) for i in range(B)])
                         .astype(np.complex64)).to(dev)
    u = torch.from_numpy(synth.random_field(1, (B, 128, 128)).astype(np.complex64)).to(dev)
    t = torch.from_numpy(synth.random_field(2, (B, 128, 128)).astype(np.complex64)).to(dev)
    out = torch.empty_like(u)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        net.forward(f, u, out)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.reps):
        net.forward(f, u, out)
    e1.record()
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1) / args.reps
    for _ in range(2):
        net.train_step(f, u, t, 1e-4)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.reps):
        net.train_step(f, u, t, 1e-4)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"batch": B, "inference_ms": fwd, "train_step_ms": e0.elapsed_time(e1) / args.reps}))
    net.close()


if __name__ == "__main__":
    main()
