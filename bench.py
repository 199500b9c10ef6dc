#!/usr/bin/env python
"""Throughput of the CISOR hot path on one GB300 (or N independent replicas).

Workload (default): 256 x 256 grid at lambda/8 (FFT padded to 512 x 512), 64
plane-wave transmitters, 256 receivers on a circle of radius 24 lambda, 10
seeded random ellipses with contrast up to 1.0 plus 0.05i absorption, 40 dB
noise.  One step is one relaxed-FISTA iteration (Eqs. 9-11) from a fixed
state: 64 forward field solves and 64 adjoint field solves (Eq. 13), each from
a cold start to true relative residual 1e-4, sensing and adjoint sensing, the
gradient (Prop. 1), the FGP TV prox and the momentum update.  The metric
counts LS field solves (forward + adjoint) per second.

``--config c3`` runs the 3D workload instead: 64^3 voxels at lambda/6 (FFT
128^3), 48 plane waves over the upper hemisphere, 1024 receivers on a plane,
5 seeded random spheres with contrast up to 0.3.  ``--config c7`` runs the 3D
vectorial model of the appendix (32^3 voxels, 81 polarised plane waves, 36
receivers measuring E_z).  ``--config c6`` runs a
Fresnel-style 2D set-up: 8 line sources, 360 receivers of which each source
records the 240 farther than 60 degrees from it.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LS field solves/s at residual 1e-4, learned vs cold start; % of HBM peak"
UNIT = "solves/s"


def _fp32_peak(device):
    """FP32 FMA peak of the device from its attributes: SMs x FP32 lanes per SM x 2 flops x peak SM clock."""
    from paper_1708_01663_gb300 import cisor
    d = cisor.device_info(device)
    lanes = d["fp32_lanes"] or 128
    tf = d["sm_count"] * lanes * 2 * d["max_clock_khz"] * 1e3 / 1e12
    return tf, {"sm_count": d["sm_count"], "fp32_lanes_per_sm": lanes, "max_sm_clock_mhz": d["max_clock_khz"] / 1e3,
                "cc": d["cc"], "source": "cudaDeviceGetAttribute (MultiProcessorCount, ClockRate) via cisor_device_info"}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cisor", choices=["cisor", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--max-iter", type=int, default=5000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tx-chunk", type=int, default=-1,
                    help="transmitters per convolution launch instead of the autotuned chunk (0: all at once)")
    ap.add_argument("--fno-train", type=int, default=2000, help="c4: training phantoms (32 samples each)")
    ap.add_argument("--fno-minutes", type=float, default=2.0, help="c4: training time budget")
    ap.add_argument("--cols-cta", type=int, default=0, choices=[0, 16, 256, 512],
                    help="column-kernel shape instead of autotuning it (0: autotune); for launch lists "
                         "taken under a profiler, whose replays change the autotuner's timings")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(",") for r in self.tmp.read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for nm, v in zip(names, r[4:8]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _state0(f_true):
    """Fixed starting point of the timed step: 0.9 x the phantom (inside the box)."""
    s0 = 0.9 * f_true
    return np.ascontiguousarray(s0, dtype=np.complex64)


def _oracle_sample_solves(cfg, f_point, angles, rx, txs, tol):
    """Cold-start FP64 oracle forward solves of the given transmitters; returns (solves, seconds, note, fields)."""
    from oracle import model, solve
    n, dim = cfg["n"], cfg["dim"]
    if cfg.get("vectorial"):
        from oracle import vector
        tx = np.asarray(angles)[list(txs)]
        prob = vector.VectorProblem(n, cfg["delta"], tx[:, :3], tx[:, 3:], rx)
        t0 = time.perf_counter()
        xs = vector.solve_fields(prob, f_point, prob.u_in, tol)
        sec = time.perf_counter() - t0
        return len(txs), sec, (f"{len(txs)} cold-start vectorial forward solves (transmitters {txs[0]}-{txs[-1]}) "
                               f"to residual {tol:g}, FP64 numpy BiCGSTAB, {sec:.1f} s"), list(xs)
    shape = (n,) * dim
    prob = model.Problem(n, cfg["delta"], np.asarray(angles)[list(txs)], rx, dim=dim,
                         tx_kind=cfg.get("tx_kind", "plane"))
    apply = lambda v: prob.A(f_point, v.reshape(shape)).ravel()
    t0 = time.perf_counter()
    xs = [solve.bicgstab(apply, prob.u_in[t].ravel(), prob.u_in[t].ravel(), tol, 20000)[0]
          for t in range(len(txs))]
    sec = time.perf_counter() - t0
    return len(txs), sec, (f"{len(txs)} cold-start forward solves (transmitters {txs[0]}-{txs[-1]}) to residual "
                           f"{tol:g}, FP64 numpy BiCGSTAB, {sec:.1f} s"), [x.reshape(shape) for x in xs]


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_worker(cfg_name, txs, tol, rounds, barrier, queue):
    """One host process of the oracle baseline (spawned): for each of its transmitters builds the
    single-transmitter FP64 problem and its measurements (untimed), then runs `rounds` timed rounds,
    each a cold-start forward solve, residual, adjoint solve and gradient term (Prop. 1) per transmitter
    to residual `tol`; every round starts at a barrier shared by all workers."""
    from oracle import grad, model, vector
    from paper_1708_01663_gb300 import synth
    cfg, f_true, angles, rx = synth.make_inputs(cfg_name)
    n, dim = cfg["n"], cfg["dim"]
    s0 = _state0(f_true).astype(np.complex128)
    ft = f_true.astype(np.complex128)
    items = []
    for t in txs:
        noise = synth.complex_noise(cfg["seed"] + 100, (cfg["T"], cfg["M"]))[t]
        if cfg.get("vectorial"):
            tx = np.asarray(angles)[[t]]
            prob = vector.VectorProblem(n, cfg["delta"], tx[:, :3], tx[:, 3:], rx)
            u = vector.solve_fields(prob, ft, prob.u_in, 1e-6)
            y = prob.sense(ft, u)
        else:
            prob = model.Problem(n, cfg["delta"], np.asarray(angles)[[t]], rx, dim=dim,
                                 tx_kind=cfg.get("tx_kind", "plane"))
            _, y, _, _ = grad.forward(prob, ft, 1e-6)
        mask = cfg["rx_mask"][[t]] if "rx_mask" in cfg else None
        y = y + np.linalg.norm(y) * 10 ** (-cfg["snr_db"] / 20) / np.sqrt(y.size) * noise[None]
        items.append((prob, y, mask))
    for _ in range(rounds):
        barrier.wait()
        t0 = time.perf_counter()
        for prob, y, mask in items:
            if cfg.get("vectorial"):
                vector.data_and_grad(prob, s0, y, tol)
            else:
                grad.data_and_grad(prob, s0, y, tol, mask=mask)
        queue.put((t0, time.perf_counter()))


def _oracle_rounds(cfg_name, T, tol, rounds, workers=None):
    """Timed rounds of the oracle baseline on the host cores: one spawned process per core, one
    transmitter each (the first `workers` transmitters); returns (per-round wall seconds, workers)."""
    import multiprocessing as mp
    workers = max(1, min(workers or (os.cpu_count() or 1), T))
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers)
    queue = ctx.Queue()
    procs = _spawn_single_threaded(ctx, _oracle_worker,
                                   [(cfg_name, [w], tol, rounds, barrier, queue) for w in range(workers)])
    walls = []
    for _ in range(rounds):
        marks = [queue.get(timeout=3600) for _ in range(workers)]
        walls.append(max(m[1] for m in marks) - min(m[0] for m in marks))
    for p in procs:
        p.join()
        if p.exitcode != 0:
            raise RuntimeError(f"oracle worker exited with {p.exitcode}")
    return walls, workers


def _oracle_sample_note(cfg_name, cfg, workers, tol):
    what = ("vectorial forward + adjoint solves and gradient term" if cfg.get("vectorial")
            else "forward + adjoint solves and gradient term (Prop. 1)")
    return (f"FP64 numpy oracle, {workers} spawned processes on {workers} host cores ({_cpu_model()}), one "
            f"transmitter each (transmitters 0-{workers - 1} of {cfg['T']}): cold-start {what} at the step's "
            f"state to residual {tol:g}; measurements from the oracle's own forward model of the phantom "
            f"(residual 1e-6) plus 40 dB noise per transmitter; set-up untimed, rounds started at a barrier")


def _graddiv_torch(C, delta):
    """Comparison only: the appendix's finite-difference grad-div of [B, 3, n, n, n] fields (zero outside)."""
    import torch
    P = torch.nn.functional.pad(C, (1, 1, 1, 1, 1, 1))
    n = C.shape[-1]
    ax = {0: -1, 1: -2, 2: -3}

    def sh(a, offs):
        sl = [slice(1, n + 1)] * 3
        for comp, o in offs.items():
            sl[3 + ax[comp]] = slice(1 + o, n + 1 + o)
        return a[(Ellipsis,) + tuple(sl)]

    out = []
    for c in range(3):
        acc = (sh(P[:, c], {c: 1}) - 2 * sh(P[:, c], {}) + sh(P[:, c], {c: -1})) / delta ** 2
        for j in range(3):
            if j != c:
                acc = acc + (sh(P[:, j], {c: -1, j: -1}) - sh(P[:, j], {c: -1, j: 1}) - sh(P[:, j], {c: 1, j: -1})
                             + sh(P[:, j], {c: 1, j: 1})) / (4 * delta ** 2)
        out.append(acc)
    return torch.stack(out, 1)


def _cufft_matvec_ms(ctx, f_dev, x_dev, dim, reps=20, vectorial=False, delta=1.0, k=2 * np.pi):
    """Comparison only (never on the product path): the same batched A x with torch.fft (cuFFT):
    zero-pad f x to P^d, FFT, times the library's own spectrum, inverse FFT, crop, subtract
    (vectorial: per component, then the grad-div stencil)."""
    import torch
    P, n = ctx.P, ctx.n
    gh = torch.empty((P,) * dim, dtype=torch.complex64, device=x_dev.device)
    ctx.green_spectrum(gh)
    axes = tuple(range(-dim, 0))
    crop = (Ellipsis,) + (slice(0, n),) * dim
    pad = torch.zeros(x_dev.shape[:-dim] + (P,) * dim, dtype=torch.complex64, device=x_dev.device)

    def once():
        pad[crop] = f_dev * x_dev
        y = torch.fft.ifftn(torch.fft.fftn(pad, dim=axes) * gh, dim=axes)[crop]
        if vectorial:
            return x_dev - y - _graddiv_torch(y, delta) / k ** 2
        return x_dev - y

    for _ in range(3):
        once()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _workload(name, cfg):
    T, M = cfg["T"], cfg["M"]
    if cfg.get("vectorial"):
        return (f"{name}: 3D vectorial (appendix), 32^3 voxels at lambda/16, FFT 64^3 per component, {T} polarised "
                f"plane waves over the upper hemisphere, {M} Rx measuring E_z on a circle of {cfg['rx_radius']} lambda, "
                f"receivers within {cfg['rx_min_deg']:.0f} deg masked off, 2 spheres contrast<=1.5, 40 dB")
    if cfg.get("tx_kind") == "point":
        return (f"{name}: Fresnel-style 2D, 128x128 over 1.5 lambda, FFT 256x256, {T} line sources at "
                f"{cfg['tx_radius']} lambda, {M} Rx at {cfg['rx_radius']} lambda, receivers within "
                f"{cfg['rx_min_deg']:.0f} deg of the source masked off, 3 ellipses contrast<=1.0, 40 dB")
    if cfg["dim"] == 3:
        return (f"{name}: 64^3 voxels at lambda/6, FFT 128^3, {T} plane waves over the upper hemisphere, "
                f"{M} Rx on a plane, 5 spheres contrast<=0.3, 40 dB")
    return f"{name}: 256x256 grid at lambda/8, FFT 512x512, {T} Tx, {M} Rx, 10 ellipses contrast<=1.0+0.05i, 40 dB"


def run_reference(args):
    """The FP64 oracle as the reference arm: each step is one barrier-started round of cold-start
    forward + adjoint solves (and the gradient term), one transmitter per host core."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_1708_01663_gb300 import synth
    cfg = synth.make_inputs(args.config)[0]
    walls, workers = _oracle_rounds(args.config, cfg["T"], args.tol, args.warmup + args.steps)
    timed = walls[args.warmup:]
    total = sum(timed)
    value = 2 * workers * len(timed) / total
    note = _oracle_sample_note(args.config, cfg, workers, args.tol)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload(args.config, cfg), "sample": note,
                   "solves_per_step": 2 * workers, "same_config": True},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": note},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def conv_sources_hash():
    """Hash of the sources of the convolution kernels (conv.cu, conv_cluster.cu, regfft.cuh, fft.cuh, dots.cuh)."""
    h = hashlib.sha256()
    for name in ("conv.cu", "conv_cluster.cu", "regfft.cuh", "fft.cuh", "dots.cuh"):
        with open(os.path.join(ROOT, "paper_1708_01663_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_summary(config):
    """ncu DRAM bytes per matvec pass from profiles/, valid only while the kernels are unchanged."""
    path = os.path.join(ROOT, "profiles", f"conv_matvec_{config}.md")
    try:
        with open(path) as fh:
            text = fh.read()
        vals = {}
        for line in text.splitlines():
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                v = v.strip()
                vals[k.strip()] = v.split("`")[1] if v.startswith("`") and v.count("`") >= 2 else v
        if vals.get("conv_sources_sha256_16") != conv_sources_hash():
            return None
        return float(vals["dram_bytes_per_pass"])
    except Exception:
        return None


def run_c4(args):
    """Learned vs cold start on the FNO workload: 128 x 128 grids at lambda/8 (FFT 256), 32 plane waves,
    phantoms of 3-10 seeded ellipses with real contrast in [0, 0.8].  The network is trained first
    (solver-generated fields of --fno-train phantoms, Adam for --fno-minutes; untimed); each timed step is
    one held-out phantom solved twice to residual 1e-4: from the cold start (x0 = u_in) and from the
    learned warm start (x0 = u_in + FNO(f, u_in), inference inside the timed region).  value = learned
    solves/s; the cold figure sits beside it."""
    import torch

    from paper_1708_01663_gb300 import build, cisor, train_fno
    build.build()
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    T, n = train_fno.T, train_fno.N
    ang, rx = train_fno.geometry()
    ctx = cisor.Cisor(n, train_fno.DELTA, ang, rx)
    cols_nt = ctx.autotune(reps=10)
    t0 = time.time()
    fs, usc, u_in = train_fno.generate(ctx, range(args.fno_train), dev)
    t_gen = time.time() - t0
    net = cisor.FNO(max_batch=T, seed=1714)
    t0 = time.time()
    steps, losses = train_fno.train(net, fs, usc, u_in, args.fno_minutes)
    t_train = time.time() - t0
    del fs, usc
    u = torch.empty((T, n * n), dtype=torch.complex64, device=dev)
    x0 = torch.empty_like(u)
    held = list(range(100000, 100000 + args.warmup + args.steps))
    fph = [torch.from_numpy(train_fno.phantom(i).astype(np.complex64).ravel()).to(dev) for i in held]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    cold_ms, warm_ms, inf_ms, ci, wi, pred = [], [], [], [], [], []
    clocks = ClockSampler(local)
    l0 = 0
    for k, f in enumerate(fph):
        if k == args.warmup:
            torch.cuda.synchronize()
            clocks.start()
            l0 = ctx.launch_count()
        ev[0].record()
        _, ic = ctx.forward(f, u_out=u, tol=args.tol, max_iter=args.max_iter, x0_mode=0, check=False)
        ev[1].record()
        u_ref = u.clone()
        ev[2].record()
        net.warm_start(ctx, f, x0)
        ev[3].record()
        torch.cuda.synchronize()
        t_inf = ev[2].elapsed_time(ev[3])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        net.warm_start(ctx, f, x0)
        _, iw = ctx.forward(f, x0=x0, u_out=u, tol=args.tol, max_iter=args.max_iter, x0_mode=1, check=False)
        e1.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            cold_ms.append(ev[0].elapsed_time(ev[1]))
            warm_ms.append(e0.elapsed_time(e1))
            inf_ms.append(t_inf)
            ci.append(ic.iters_mean)
            wi.append(iw.iters_mean)
            pred.append(float(torch.linalg.vector_norm(x0 - u_ref) / torch.linalg.vector_norm(u_ref - u_in)))
    clk = clocks.stop()
    launches = ctx.launch_count() - l0
    value = T * len(warm_ms) / (sum(warm_ms) / 1e3)
    cold_value = T * len(cold_ms) / (sum(cold_ms) / 1e3)
    # end to end through host buffers: f from pinned host memory, warm start, solve, fields back to the host
    f_h = [f.cpu().pin_memory() for f in fph[:args.steps]]
    u_h = torch.empty((T, n * n), dtype=torch.complex64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for f in f_h:
        fd = f.to(dev, non_blocking=True)
        net.warm_start(ctx, fd, x0)
        ctx.forward(fd, x0=x0, u_out=u_h, tol=args.tol, max_iter=args.max_iter, x0_mode=1, check=False)
    torch.cuda.synchronize()
    e2e = T * len(f_h) / (time.perf_counter() - t0)
    mv_ms = ctx.time_matvec(fph[0], adjoint=False, reps=20)
    Pd = ctx.P ** 2
    alg_flops = T * 2 * 5 * Pd * np.log2(Pd)
    alg_bytes = T * 16 * ctx.N + 8 * ctx.N
    fp32_peak, peak_inputs = _fp32_peak(local)
    hbm_peak, peak_kind = _peaks()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": len(warm_ms), "warmup": args.warmup,
        "ms_per_step": float(np.mean(warm_ms)), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 (FNO: bf16 weights, fp32 accumulate)", "data": "synthetic",
        "config": {"workload": "c4: 128x128 at lambda/8, FFT 256x256, 32 plane waves, 64 Rx, 3-10 ellipses "
                               "contrast [0, 0.8]; learned warm start (FNO: 4 Fourier layers, width 32, 16 modes)",
                   "step": "one held-out phantom: 32 solves to residual 1e-4 from the learned warm start, "
                           "inference included",
                   "train_phantoms": args.fno_train, "train_samples": args.fno_train * T, "gen_s": t_gen,
                   "train_s": t_train, "train_steps": steps, "loss_first": float(np.mean(losses[:20])),
                   "loss_last": float(np.mean(losses[-50:])), "heldout_phantoms": len(warm_ms),
                   "pred_rel_err_mean": float(np.mean(pred)), "cols_cta": cols_nt,
                   "l2": "working set < L2: each timed phantom follows the previous phantom's solves"},
        "learned_vs_cold": {"learned_solves_per_s": value, "cold_solves_per_s": cold_value,
                            "time_saved_frac": 1.0 - float(np.mean(warm_ms)) / float(np.mean(cold_ms)),
                            "cold_ms_per_phantom": float(np.mean(cold_ms)),
                            "learned_ms_per_phantom": float(np.mean(warm_ms)),
                            "inference_ms_per_phantom": float(np.mean(inf_ms)),
                            "cold_iters_mean": float(np.mean(ci)), "learned_iters_mean": float(np.mean(wi)),
                            "iters_saved_frac": 1.0 - float(np.mean(wi)) / float(np.mean(ci)),
                            "cold_iters_p95": float(np.percentile(ci, 95)),
                            "learned_iters_p95": float(np.percentile(wi, 95))},
        "roofline": {"bound": "alu", "achieved": alg_flops / (mv_ms * 1e-3) / 1e12, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": alg_flops / (mv_ms * 1e-3) / 1e12 / fp32_peak, "traffic": None,
                     "kernel": "batched FFT matvec A x over all T", "ms_per_launch": mv_ms,
                     "peak_inputs": peak_inputs,
                     "hbm": {"achieved": alg_bytes / (mv_ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                             "frac": alg_bytes / (mv_ms * 1e-3) / 1e9 / hbm_peak,
                             "peak_kind": f"{peak_kind} copy bandwidth"}},
        "cpu_baseline": None,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": n * n * 8, "d2h_bytes_per_step": T * n * n * 8},
        "gpu_launches": launches, "clocks": clk,
    }
    if not args.no_cpu_baseline:
        walls, workers = _oracle_rounds_c4(args.tol)
        line["cpu_baseline"] = {"value": workers * len(walls) / sum(walls), "unit": UNIT, "cores": workers,
                                "kind": "oracle",
                                "sample": f"FP64 numpy oracle, {workers} spawned processes on {workers} host cores "
                                          f"({_cpu_model()}): cold-start forward solves of held-out phantom 0, one "
                                          f"transmitter per process, to residual {args.tol:g}; {len(walls)} rounds"}
    print(json.dumps(line), flush=True)
    net.close()
    ctx.close()


def _c4_worker(t, tol, rounds, barrier, queue):
    from oracle import grad, model
    from paper_1708_01663_gb300 import train_fno
    ang, rx = train_fno.geometry()
    prob = model.Problem(train_fno.N, train_fno.DELTA, np.asarray(ang)[[t]], rx)
    f = train_fno.phantom(100000).astype(np.complex128)
    for _ in range(rounds):
        barrier.wait()
        t0 = time.perf_counter()
        grad.forward(prob, f, tol)
        queue.put((t0, time.perf_counter()))


def _spawn_single_threaded(ctx, target, argsets):
    """Start one spawned process per argument tuple with one BLAS / OpenMP thread each."""
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"  # one thread per process: the processes are the parallelism
    try:
        procs = [ctx.Process(target=target, args=a) for a in argsets]
        for p in procs:
            p.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return procs


def _oracle_rounds_c4(tol, rounds=3):
    import multiprocessing as mp
    from paper_1708_01663_gb300 import train_fno
    workers = max(1, min(os.cpu_count() or 1, train_fno.T))
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(workers), ctx.Queue()
    procs = _spawn_single_threaded(ctx, _c4_worker, [(w, tol, rounds, barrier, queue) for w in range(workers)])
    walls = []
    for _ in range(rounds):
        marks = [queue.get(timeout=3600) for _ in range(workers)]
        walls.append(max(m[1] for m in marks) - min(m[0] for m in marks))
    for p in procs:
        p.join()
    return walls, workers


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.config == "c4":
        run_c4(args)
        return
    ws, rank, local = _dist()
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1708_01663_gb300 import build, cisor, shard, synth
    build.build()
    dev = torch.device("cuda", local)
    cfg, f_true, angles, rx = synth.make_inputs(args.config)
    n, T, M, dim = cfg["n"], cfg["T"], cfg["M"], cfg["dim"]
    complex_f = cfg["imag"] != 0.0
    vec = bool(cfg.get("vectorial"))
    # N > 1: weak scaling by transmitter shards.  One reconstruction with N x T plane waves at uniform
    # angles; rank r solves its contiguous block of T and the ranks all-reduce g and D once per step.
    sharded = ws > 1 and dim == 2 and cfg.get("tx_kind", 0) in (0, "plane") and not vec
    T_total = T * ws if sharded else T
    if sharded:
        angles = synth.plane_wave_angles(T_total)[rank * T:(rank + 1) * T]
    ctx = cisor.Cisor(n, cfg["delta"], angles, rx, complex_f=complex_f, dim=dim, tx_kind=cfg.get("tx_kind", 0),
                      vectorial=vec)
    if "rx_mask" in cfg:
        ctx.set_rx_mask(cfg["rx_mask"])
    if args.cols_cta:
        ctx.set_cols_cta(args.cols_cta)
        ctx.set_tx_chunk(max(args.tx_chunk, 0))
    else:
        ctx.autotune(reps=10)  # pick the column-kernel shape and transmitter chunk by measurement
        if args.tx_chunk >= 0:
            ctx.set_tx_chunk(args.tx_chunk)
    cols_nt, tx_chunk = ctx.tuning()

    # synthetic measurements: GPU forward model of the phantom + seeded 40 dB noise (untimed set-up)
    f_dev = torch.from_numpy(np.ascontiguousarray(f_true, dtype=np.complex64)).to(dev)
    y_dev = torch.empty((T, M), dtype=torch.complex64, device=dev)
    ctx.forward(f_dev, y_out=y_dev, tol=1e-6, max_iter=args.max_iter, check=False)
    torch.cuda.synchronize()
    noise = synth.complex_noise(cfg["seed"] + 100, (T_total, M)).astype(np.complex64)
    noise = torch.from_numpy(noise[rank * T:(rank + 1) * T] if sharded else noise).to(dev)
    ny2 = torch.tensor([float(torch.linalg.vector_norm(y_dev)) ** 2], dtype=torch.float64, device=dev)
    if sharded:
        dist.all_reduce(ny2)
    sigma = float(ny2.item()) ** 0.5 * 10 ** (-cfg["snr_db"] / 20) / np.sqrt(T_total * M)
    y_dev += sigma * noise
    H_dev = torch.empty((M, ctx.Nf), dtype=torch.complex64, device=dev)
    ctx.sensing_matrix(H_dev)
    u_in = torch.empty((T, ctx.Nf), dtype=torch.complex64, device=dev)
    ctx.incident(u_in)
    # L_Born <= T max|u_in|^2 ||H||_F^2 (max |u_in| = 1 for plane waves)
    gamma = 1.0 / (T_total * float(u_in.abs().max()) ** 2 * float(torch.linalg.vector_norm(H_dev)) ** 2)
    del H_dev, u_in

    s0 = torch.from_numpy(_state0(f_true)).to(dev)
    f_st = torch.empty_like(s0)
    s_st = torch.empty_like(s0)
    state = ctx.new_state(f_st, s_st, cfg["alpha"], gamma, cfg["tau"], cfg["tv_iters"], 0.0, 2.0, 0.0, 0.5)

    infos = []
    iters_all = []

    g_red = torch.empty_like(s0)  # the all-reduced gradient of a sharded step

    def step(st, y, f_buf, s_buf):
        f_buf.copy_(s0) if hasattr(f_buf, "copy_") else None
        s_buf.copy_(s0) if hasattr(s_buf, "copy_") else None
        st.t, st.k = 1.0, 1
        if sharded:  # this rank's gradient, NCCL all-reduce of g and D, redundant update (Eqs. 9-11)
            _, info = shard.sharded_step(ctx, st, s_buf, y, g_red, tol=args.tol, max_iter=args.max_iter, x0_mode=0,
                                         check=False)
        else:
            _, info = ctx.step(st, y, tol=args.tol, max_iter=args.max_iter, x0_mode=0, check=False)
        infos.append(info.as_dict())
        iters_all.extend(ctx.solve_iterations(False).tolist() + ctx.solve_iterations(True).tolist())

    for _ in range(args.warmup):
        step(state, y_dev, f_st, s_st)
    torch.cuda.synchronize()
    infos.clear()
    iters_all.clear()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = ctx.launch_count()
    # Working sets smaller than twice L2 (129 MB) are timed step by step with an
    # L2 flush (a 512 MB write) between the steps, outside the timed windows;
    # larger ones stream through L2 by themselves and are timed back to back.
    working = 12 * T * ctx.Nf * 8 + M * ctx.Nf * 8
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev) if working < 2 * (129 << 20) else None
    if flush is None:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            step(state, y_dev, f_st, s_st)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
    else:
        ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step(state, y_dev, f_st, s_st)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
    launches = ctx.launch_count() - l0
    clk = clocks.stop()
    if dist:
        dist.barrier()
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    step_infos = list(infos)
    solves_per_step = 2 * T
    value = ws * solves_per_step * args.steps / (ms / 1e3)

    # end to end through host (pinned) buffers: H2D of y and the state, D2H of the new state
    y_h = torch.empty((T, M), dtype=torch.complex64, pin_memory=True)
    y_h.copy_(y_dev.cpu())
    s0_h = s0.cpu()
    f_h = torch.empty_like(s0_h).pin_memory()
    s_h = torch.empty_like(s0_h).pin_memory()
    st_h = ctx.new_state(f_h, s_h, cfg["alpha"], gamma, cfg["tau"], cfg["tv_iters"], 0.0, 2.0, 0.0, 0.5)

    def step_h():
        f_h.copy_(s0_h)
        s_h.copy_(s0_h)
        st_h.t, st_h.k = 1.0, 1
        if sharded:
            shard.sharded_step(ctx, st_h, s_h, y_h, g_red, tol=args.tol, max_iter=args.max_iter, x0_mode=0,
                               check=False)
        else:
            ctx.step(st_h, y_h, tol=args.tol, max_iter=args.max_iter, x0_mode=0, check=False)

    step_h()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_h()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = ws * solves_per_step * args.steps / e2e_s
    h2d = y_h.numel() * 8 + 2 * s0_h.numel() * 8
    d2h = 2 * s0_h.numel() * 8

    # roofline of the dominant kernel chain: one batched FFT matvec over all T transmitters,
    # timed with CUDA events on the library's own stream (cisor_time_matvec)
    mv_ms = ctx.time_matvec(s0, adjoint=False, reps=20)
    N = ctx.N
    Pd = ctx.P ** dim
    ncomp = 3 if vec else 1
    alg_bytes = T * 16 * ctx.Nf + 8 * N                  # read x, write y per transmitter, f once
    alg_flops = ncomp * T * 2 * 5 * Pd * np.log2(Pd)     # forward + inverse P^d FFT per field component (unpruned)
    achieved_tf = alg_flops / (mv_ms * 1e-3) / 1e12
    achieved_gbs = alg_bytes / (mv_ms * 1e-3) / 1e9
    hbm_peak, peak_kind = _peaks()
    fp32_peak, peak_inputs = _fp32_peak(local)
    traffic = _traffic_summary(args.config)
    fshape = (T, 3) + (n,) * dim if vec else (T,) + (n,) * dim
    u_in = torch.empty(fshape, dtype=torch.complex64, device=dev)
    ctx.incident(u_in)
    cufft_ms = _cufft_matvec_ms(ctx, s0, u_in, dim, vectorial=vec, delta=cfg["delta"], k=2 * np.pi)
    del u_in

    cpu = None
    field_err = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        s0n = _state0(f_true).astype(np.complex128)
        walls, workers = _oracle_rounds(args.config, T, args.tol, 2)
        note = _oracle_sample_note(args.config, cfg, workers, args.tol) + f"; {len(walls)} rounds"
        cpu = {"value": 2 * workers * len(walls) / sum(walls), "unit": UNIT, "cores": workers, "kind": "oracle",
               "sample": note}
        # error of the converged field (GPU, residual tol) against a tight FP64 oracle solve of transmitter 0
        _, _, _, ref = _oracle_sample_solves(cfg, s0n, angles, rx, [0], 1e-9)
        u_dev = torch.empty((T, 3) + (n,) * dim if vec else (T,) + (n,) * dim, dtype=torch.complex64, device=dev)
        ctx.forward(s0, u_out=u_dev, tol=args.tol, max_iter=args.max_iter, check=False)
        u0 = u_dev[0].cpu().numpy().astype(np.complex128)
        field_err = {"rel_l2": float(np.linalg.norm(u0 - ref[0]) / np.linalg.norm(ref[0])),
                     "what": f"transmitter 0 at the step's state, GPU solve to residual {args.tol:g} vs FP64 "
                             "oracle solve to residual 1e-9"}

    if rank == 0:
        it_f = [i["iters_mean"] for i in step_infos]
        it_a = [i["adj_iters_mean"] for i in step_infos]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": _workload(args.config, dict(cfg, T=T_total)) + (
                           f" ({T} per rank)" if sharded else ""),
                       "step": "one relaxed-FISTA iteration from a fixed state: T forward + T adjoint "
                               "cold-start solves to residual 1e-4, sensing, gradient, FGP prox (20 it)",
                       "solves_per_step": solves_per_step, "start": "cold (u_in / 0)",
                       "l2": (f"working set > L2 (Krylov vectors 12 x {T * N * 8 / 2**20:.0f} MB)" if flush is None
                              else "L2 flushed between timed steps (512 MB write outside the timed windows)"),
                       "parallelism": (f"transmitter shards: {ws} ranks x {T} of {T_total} plane waves, NCCL "
                                       "all-reduce of g and D per step, redundant prox and momentum") if sharded
                                      else ("independent replicas" if ws > 1 else "single GPU"),
                       "cols_cta": cols_nt, "cols_cta_from": "flag" if args.cols_cta else "autotune",
                       "tx_chunk": tx_chunk,
                       "tx_chunk_from": "flag" if (args.cols_cta or args.tx_chunk >= 0) else "autotune",
                       "fwd_iters_mean": float(np.mean(it_f)) if it_f else None,
                       "fwd_iters_max": max(i["iters_max"] for i in step_infos) if step_infos else None,
                       "adj_iters_max": max(i["adj_iters_max"] for i in step_infos) if step_infos else None,
                       "adj_iters_mean": float(np.mean(it_a)) if it_a else None,
                       "resid_max": max(i["resid_max"] for i in step_infos) if step_infos else None,
                       "not_converged": sum(i["n_not_converged"] for i in step_infos),
                       "iters_p95": float(np.percentile(iters_all, 95)) if iters_all else None,
                       "field_err_vs_oracle": field_err},
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved_tf / fp32_peak, "traffic": traffic,
                         "kernel": "batched FFT matvec A x over all T (conv_rows_fwd + conv_cols + conv_rows_inv)"
                                   if dim == 2 else "batched FFT matvec A x over all T (conv_rows_fwd + conv_cols "
                                   "y-forward + conv_cols z-spectrum + conv_cols y-inverse + conv_rows_inv"
                                   + (" per field component, + the grad-div stencil)" if vec else ")"),
                         "ms_per_launch": mv_ms, "alg_flops_per_launch": alg_flops,
                         "alg_bytes_per_launch": alg_bytes,
                         "peak_kind": "FP32 FMA peak from the device's attributes: SMs x FP32 lanes per SM x 2 "
                                      "flops x peak SM clock",
                         "peak_inputs": peak_inputs,
                         "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": achieved_gbs / hbm_peak, "peak_kind": f"{peak_kind} copy bandwidth",
                                 "what": "algorithmic bytes (read x, write A x per transmitter, f once) / CUDA-event "
                                         "time of one pass",
                                 "dram_achieved": (traffic / (mv_ms * 1e-3) / 1e9) if traffic else None,
                                 "dram_frac": (traffic / (mv_ms * 1e-3) / 1e9 / hbm_peak) if traffic else None,
                                 "dram_what": "ncu DRAM bytes of one pass (profiles/, cold cache) / CUDA-event time "
                                              "of one pass; null when the kernels changed since the capture"}},
            "comparison": {"cufft_matvec_ms": cufft_ms, "cisor_matvec_ms": mv_ms,
                           "what": "the same batched A x over all T with torch.fft (cuFFT: pad, FFT, x ghat, IFFT, "
                                   "crop) on the same inputs; timed for comparison only, not on the product path"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
