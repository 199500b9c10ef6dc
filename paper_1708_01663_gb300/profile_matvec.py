"""Time (and give a profiler something small to capture) one batched FFT matvec.

    python -m paper_1708_01663_gb300.profile_matvec --config c2 --reps 3

Builds the tables of a named workload (seeded phantom, all transmitters, or
the first ``--T``), autotunes the column-kernel shape (2 or 3 variants x
(1 + 5) passes) and runs one untimed plus ``reps`` timed passes of
y_t = A x_t over every transmitter through cisor_time_matvec.
``--cols-cta 512|256|16|8`` sets the column-kernel shape instead of measuring
it (16: the two-stage kernel, 8: the one-kernel cluster pass; ``--tx-chunk``
the transmitter chunk), so that no convolution runs
before the untimed pass and
``ncu --clock-control none --metrics gpu__time_duration.sum -k regex:conv_ -c k``
(k = 3 kernels per pass in 2D, 5 in 3D) lists exactly that pass; a full-metric
capture names one kernel (``-k regex:conv_cols``) and one launch (``-c 1``).
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c2")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--adjoint", action="store_true")
    ap.add_argument("--T", type=int, default=None)
    ap.add_argument("--cols-cta", type=int, default=0, choices=[0, 8, 16, 256, 512])
    ap.add_argument("--tx-chunk", type=int, default=0)
    args = ap.parse_args()
    import torch

    from paper_1708_01663_gb300 import build, cisor, synth
    build.build()
    cfg, f, angles, rx = synth.make_inputs(args.config, T=args.T)
    ctx = cisor.Cisor(cfg["n"], cfg["delta"], angles, rx, complex_f=cfg["imag"] != 0.0, dim=cfg["dim"],
                      tx_kind=cfg.get("tx_kind", 0), vectorial=bool(cfg.get("vectorial")))
    fd = torch.from_numpy(np.ascontiguousarray(0.9 * f, dtype=np.complex64)).cuda()
    if args.cols_cta:
        ctx.set_cols_cta(args.cols_cta)
        ctx.set_tx_chunk(args.tx_chunk)
        cols = args.cols_cta
    else:
        cols = ctx.autotune(reps=5)  # column-FFT CTA size chosen by measurement
    ms = ctx.time_matvec(fd, adjoint=args.adjoint, reps=args.reps)
    N = ctx.N
    alg = cfg["T"] * 16 * N + 8 * N
    print(json.dumps({"config": args.config, "T": cfg["T"], "n": cfg["n"], "P": ctx.P, "cols_cta": cols,
                      "ms_per_pass": ms,
                      "alg_bytes": alg, "alg_GBps": alg / ms / 1e6}))
    ctx.close()


if __name__ == "__main__":
    main()
