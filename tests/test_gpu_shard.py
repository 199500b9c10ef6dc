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
