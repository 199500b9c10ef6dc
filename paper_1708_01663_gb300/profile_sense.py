"""Time (and give a profiler something small to capture) the sensing GEMMs.

    python -m paper_1708_01663_gb300.profile_sense --config c3 [--n 32] [--reps 5]

Builds the tables of a named workload (optionally on an n^d grid instead of
the workload's own, for captures that must stay small), fills f and the
fields u with seeded random values, and runs 2 untimed and ``reps`` timed
calls of cisor_sense (Z = H (f .* u), Eq. 5) and cisor_sense_adjoint
(z = H^H w, b = conj(f) .* z, Eq. 13) on device buffers, timed with CUDA
events (each call also copies its inputs into the context's buffers).
Prints one JSON line with the times and the rates against the matrix H
that each GEMM streams (M x n^d complex64).  ``--check`` adds the relative
L2 error of both products against FP64 products of the context's own H on
the GPU (torch, complex128).  A launch list of the same
command: ``ncu --clock-control none --metrics gpu__time_duration.sum -k
regex:sense -c 20``; a full-metric capture names one kernel
(``-k regex:sense_tc_kernel``) and one or two launches, on a small ``--n``.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c3")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--check", action="store_true")
    args = ap.parse_args()
    import torch

    from paper_1708_01663_gb300 import build, cisor, synth
    build.build()
    cfg, _, tx, rx = synth.make_inputs(args.config)
    n = args.n or cfg["n"]
    ctx = cisor.Cisor(n, cfg["delta"], tx, rx, complex_f=True, dim=cfg["dim"], tx_kind=cfg.get("tx_kind", 0),
                      vectorial=bool(cfg.get("vectorial")))
    dev = torch.device("cuda", 0)
    g = torch.Generator(device="cpu").manual_seed(7)

    def crand(*shape):
        return torch.complex(torch.randn(*shape, generator=g), torch.randn(*shape, generator=g)).to(dev)

    T, M, N, Nf = ctx.T, ctx.M, ctx.N, ctx.Nf
    f = crand(N) * 0.3
    u = crand(T, Nf)
    w = crand(T, M)
    Z = torch.empty((T, M), dtype=torch.complex64, device=dev)
    z = torch.empty((T, Nf), dtype=torch.complex64, device=dev)
    b = torch.empty_like(z)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = {}
    for name, call in (("forward", lambda: ctx.sense(f, u, Z)), ("adjoint", lambda: ctx.sense_adjoint(f, w, z, b))):
        for _ in range(2):
            call()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.reps):
            call()
        e1.record()
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / args.reps
    hbytes = 8.0 * M * Nf
    flops = 8.0 * T * M * Nf
    check = {}
    if args.check:
        H = torch.empty((M, Nf), dtype=torch.complex64, device=dev)
        ctx.sensing_matrix(H)
        ctx.sense(f, u, Z)
        ctx.sense_adjoint(f, w, z, b)
        torch.cuda.synchronize()
        H64 = H.to(torch.complex128)
        Zref = (H64 @ (f.to(torch.complex128).repeat(Nf // N)[None, :] * u.to(torch.complex128)).T).T
        zref = (H64.conj().T @ w.to(torch.complex128).T).T

        def rel(a, r):
            return float(torch.linalg.vector_norm(a.to(torch.complex128) - r) / torch.linalg.vector_norm(r))
        check = {"forward_rel_err_vs_fp64": rel(Z, Zref), "adjoint_rel_err_vs_fp64": rel(z, zref)}
    print(json.dumps({"config": args.config, "n": n, "T": T, "M": M, "Nf": Nf, "H_bytes": hbytes, **check,
                      "forward_ms": times["forward"], "adjoint_ms": times["adjoint"],
                      "forward_H_GBps": hbytes / times["forward"] / 1e6,
                      "adjoint_H_GBps": hbytes / times["adjoint"] / 1e6,
                      "forward_TFLOPs": flops / times["forward"] / 1e9,
                      "adjoint_TFLOPs": flops / times["adjoint"] / 1e9}))
    ctx.close()


if __name__ == "__main__":
    main()
