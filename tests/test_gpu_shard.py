"""Transmitter sharding on one GPU: two contexts holding transmitters [0, k)
and [k, T) of one geometry.  The sum of their gradients is the full
context's (fields are solved per transmitter, so only the order of the
FP32 sum over transmitters differs), and relaxed-FISTA steps through
cisor_step_update with the summed gradient match cisor_step on the full
context and leave both shards in the same state."""
import numpy as np
import pytest

from paper_1708_01663_gb300 import build, cisor, synth
from paper_1708_01663_gb300.shard import sharded_step, tx_split
from tests.gpu_util import c64, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_two_shards_match_full_context():
    build.build()
    cfg, f_true, angles, rx = synth.make_inputs("c1")
    n, T, M = cfg["n"], cfg["T"], cfg["M"]
    full = cisor.Cisor(n, cfg["delta"], angles, rx)
    parts = [tx_split(T, 2, r) for r in range(2)]
    shards = [cisor.Cisor(n, cfg["delta"], angles[a:b], rx) for a, b in parts]
    y = np.empty((T, M), np.complex64)
    full.forward(c64(f_true), y_out=y, tol=1e-7, max_iter=3000)
    dev = torch.device("cuda")
    y_d = torch.from_numpy(y).to(dev)
    s0 = c64(0.8 * f_true)

    # gradients: sum of the shards' == the full context's
    g_full = torch.empty((n, n), dtype=torch.complex64, device=dev)
    D_full, _, _ = full.grad(torch.from_numpy(s0).to(dev), y_d, g_full, tol=1e-6, max_iter=3000)
    gs, Ds = [], []
    for (a, b), ctx in zip(parts, shards):
        g = torch.empty((n, n), dtype=torch.complex64, device=dev)
        D, _, _ = ctx.grad(torch.from_numpy(s0).to(dev), y_d[a:b].contiguous(), g, tol=1e-6, max_iter=3000)
        gs.append(g)
        Ds.append(D)
    assert abs(sum(Ds) - D_full) <= 1e-6 * D_full
    assert rel((gs[0] + gs[1]).cpu().numpy(), g_full.cpu().numpy()) < 1e-6

    # three sharded steps, the all-reduce done by a host-side sum
    gamma, tau, alpha = 0.05 / float(np.abs(g_full.cpu().numpy()).max()), cfg["tau"], cfg["alpha"]
    bufs = [(torch.from_numpy(s0).to(dev), torch.from_numpy(s0).to(dev)) for _ in shards]
    states = [ctx.new_state(f, s, alpha, gamma, tau, cfg["tv_iters"], 0.0, 2.0) for ctx, (f, s) in zip(shards, bufs)]
    ff, sf = torch.from_numpy(s0).to(dev), torch.from_numpy(s0).to(dev)
    st_full = full.new_state(ff, sf, alpha, gamma, tau, cfg["tv_iters"], 0.0, 2.0)
    gbuf = [torch.empty((n, n), dtype=torch.complex64, device=dev) for _ in shards]
    for _ in range(3):
        partial = []
        for (a, b), ctx, st, (f, s), g in zip(parts, shards, states, bufs, gbuf):
            D, _, _ = ctx.grad(s, y_d[a:b].contiguous(), g, tol=1e-6, max_iter=3000, x0_mode=2)
            partial.append((g.clone(), D))
        gsum = partial[0][0] + partial[1][0]
        Dsum = partial[0][1] + partial[1][1]
        for ctx, st, g in zip(shards, states, gbuf):
            g.copy_(gsum)
            ctx.step_update(st, g, Dsum)
        full.step(st_full, y_d, tol=1e-6, max_iter=3000, x0_mode=2)
        assert abs(Dsum - st_full.D) <= 1e-5 * st_full.D
    torch.cuda.synchronize()
    assert torch.equal(bufs[0][0], bufs[1][0]) and torch.equal(bufs[0][1], bufs[1][1])
    assert rel(bufs[0][0].cpu().numpy(), ff.cpu().numpy()) < 1e-5
    assert states[0].t == st_full.t and states[0].k == st_full.k == 4


def test_sharded_step_with_identity_reduce_is_step():
    """world size 1: sharded_step == cisor_step (same gradient, update split in two calls)."""
    build.build()
    cfg, f_true, angles, rx = synth.make_inputs("c1")
    n, T, M = cfg["n"], cfg["T"], cfg["M"]
    a = cisor.Cisor(n, cfg["delta"], angles, rx)
    b = cisor.Cisor(n, cfg["delta"], angles, rx)
    y = np.empty((T, M), np.complex64)
    a.forward(c64(f_true), y_out=y, tol=1e-7, max_iter=3000)
    dev = torch.device("cuda")
    y_d = torch.from_numpy(y).to(dev)
    s0 = c64(0.8 * f_true)
    fa, sa = torch.from_numpy(s0).to(dev), torch.from_numpy(s0).to(dev)
    fb, sb = torch.from_numpy(s0).to(dev), torch.from_numpy(s0).to(dev)
    sta = a.new_state(fa, sa, 0.96, 1e-3, 1e-3, 20, 0.0, 2.0)
    stb = b.new_state(fb, sb, 0.96, 1e-3, 1e-3, 20, 0.0, 2.0)
    g = torch.empty((n, n), dtype=torch.complex64, device=dev)
    for _ in range(2):
        a.step(sta, y_d, tol=1e-6, max_iter=3000, x0_mode=0)
        sharded_step(b, stb, sb, y_d, g, reduce=lambda g_, D: D, tol=1e-6, max_iter=3000, x0_mode=0)
    torch.cuda.synchronize()
    # D sums per-block partials with double atomics, so only its rounding may differ
    assert rel(fb.cpu().numpy(), fa.cpu().numpy()) < 1e-6 and rel(sb.cpu().numpy(), sa.cpu().numpy()) < 1e-6
    assert abs(sta.D - stb.D) <= 1e-12 * sta.D


def _shard_rank(rank, world, port, y, s0, gamma, q):
    """One rank of the two-process test: its own CUDA context (cuda:0) on its transmitter block, the
    gradient all-reduced by gloo through host memory, cisor_step_update on the summed gradient."""
    import os

    import torch.distributed as dist

    os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        cfg, f_true, angles, rx = synth.make_inputs("c1")
        a, b = tx_split(cfg["T"], world, rank)
        ctx = cisor.Cisor(cfg["n"], cfg["delta"], angles[a:b], rx)
        dev = torch.device("cuda", 0)

        def host_reduce(g, D):
            gh = torch.view_as_real(g).cpu()
            dist.all_reduce(gh)
            g.copy_(torch.view_as_complex(gh).to(dev))
            d = torch.tensor([float(D)], dtype=torch.float64)
            dist.all_reduce(d)
            return float(d.item())

        f = torch.from_numpy(s0).to(dev)
        s = torch.from_numpy(s0).to(dev)
        st = ctx.new_state(f, s, cfg["alpha"], gamma, cfg["tau"], cfg["tv_iters"], 0.0, 2.0)
        g = torch.empty_like(s)
        y_loc = torch.from_numpy(y[a:b]).to(dev)
        Ds = []
        for _ in range(3):
            sharded_step(ctx, st, s, y_loc, g, reduce=host_reduce, tol=1e-6, max_iter=3000, x0_mode=2)
            Ds.append(st.D)
        torch.cuda.synchronize()
        q.put((rank, f.cpu().numpy(), s.cpu().numpy(), Ds))
        ctx.close()
    finally:
        dist.destroy_process_group()


def test_two_processes_allreduce_match_full_context():
    """Transmitter sharding across two processes (world size 2, gloo all-reduce of g and D per step,
    each rank with its own context on the same GPU, no kernel waiting on another rank): three
    relaxed-FISTA steps leave both ranks in the state of cisor_step on the full context."""
    import multiprocessing as mp
    import socket

    build.build()
    cfg, f_true, angles, rx = synth.make_inputs("c1")
    n, T, M = cfg["n"], cfg["T"], cfg["M"]
    full = cisor.Cisor(n, cfg["delta"], angles, rx)
    y = np.empty((T, M), np.complex64)
    full.forward(c64(f_true), y_out=y, tol=1e-7, max_iter=3000)
    s0 = c64(0.8 * f_true)
    dev = torch.device("cuda")
    g_full = torch.empty((n, n), dtype=torch.complex64, device=dev)
    full.grad(torch.from_numpy(s0).to(dev), torch.from_numpy(y).to(dev), g_full, tol=1e-6, max_iter=3000)
    gamma = 0.05 / float(np.abs(g_full.cpu().numpy()).max())
    ff, sf = torch.from_numpy(s0).to(dev), torch.from_numpy(s0).to(dev)
    st_full = full.new_state(ff, sf, cfg["alpha"], gamma, cfg["tau"], cfg["tv_iters"], 0.0, 2.0)
    D_full = []
    for _ in range(3):
        full.step(st_full, torch.from_numpy(y).to(dev), tol=1e-6, max_iter=3000, x0_mode=2)
        D_full.append(st_full.D)
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, y, s0, gamma, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, f, s, Ds in res:
        assert rel(f, ff.cpu().numpy()) < 1e-5, rank
        assert rel(s, sf.cpu().numpy()) < 1e-5, rank
        assert rel(Ds, D_full) < 1e-5, rank
    assert np.array_equal(res[0][1], res[1][1])
