"""Transmitter sharding (D and Prop. 1's g are sums over transmitters) on
world-size-2 gloo process groups: the split covers every transmitter once,
and the all-reduced partial gradients of the FP64 oracle equal the full
gradient, through the same sharded_step the GPU contexts use."""
import math
import os
import socket

import numpy as np
import pytest

from paper_1708_01663_gb300.shard import tx_split

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("T,world", [(8, 2), (5, 2), (64, 3), (7, 7)])
def test_tx_split_covers_each_transmitter_once(T, world):
    parts = [tx_split(T, world, r) for r in range(world)]
    assert parts[0][0] == 0 and parts[-1][1] == T
    for (a, b), (c, d) in zip(parts, parts[1:]):
        assert b == c
    sizes = [b - a for a, b in parts]
    assert max(sizes) - min(sizes) <= 1


def test_tx_split_rejects_bad_splits():
    with pytest.raises(ValueError):
        tx_split(2, 3, 0)
    with pytest.raises(ValueError):
        tx_split(8, 2, 2)


def _problem(T):
    from oracle import model
    from paper_1708_01663_gb300 import synth
    n = 16
    angles = synth.plane_wave_angles(T)
    rx = synth.circle_receivers(8, 3.0)
    return n, angles, rx, model.Problem(n, 1.0 / 8, angles, rx)


class _OracleShard:
    """Stand-in for a rank's context: the oracle's gradient over the rank's
    transmitters and the oracle's prox + momentum as the update."""

    def __init__(self, n, angles, rx):
        from oracle import model
        self.prob = model.Problem(n, 1.0 / 8, angles, rx)

    def grad(self, s, y, g, **kw):
        from oracle import grad
        D, gr = grad.data_and_grad(self.prob, s.numpy(), y, tol=1e-12)
        g.copy_(torch.from_numpy(gr))
        return D, 0, None

    def step_update(self, st, g, D):
        from oracle import prox
        z = st["s"].numpy() - st["gamma"] * g.numpy().real
        f = prox.prox_R(z, st["gamma"] * st["tau"], 10, box_re=(-np.inf, np.inf))
        tn = (math.sqrt(4 * st["t"] ** 2 + 1) + 1) / 2
        s_new = f + st["alpha"] * (st["t"] - 1) / tn * (f - st["f"].numpy())
        st["f"].copy_(torch.from_numpy(f))
        st["s"].copy_(torch.from_numpy(s_new))
        st["t"], st["D"] = tn, D


def _rank(rank, world, port, T, out_dir):
    import torch.distributed as dist

    from paper_1708_01663_gb300 import synth
    from paper_1708_01663_gb300.shard import sharded_step
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        n, angles, rx, prob = _problem(T)
        from oracle import grad
        f_true = synth.ellipse_phantom(n, 2, (0.1, 0.4), 3)
        _, y, _, _ = grad.forward(prob, f_true, tol=1e-12)
        a, b = tx_split(T, world, rank)
        shard = _OracleShard(n, angles[a:b], rx)
        s0 = 0.5 * f_true
        st = {"f": torch.from_numpy(s0.astype(np.complex128)), "s": torch.from_numpy(s0.astype(np.complex128)),
              "t": 1.0, "alpha": 0.96, "gamma": 0.5, "tau": 1e-3, "D": None}
        g = torch.zeros((n, n), dtype=torch.complex128)
        for _ in range(2):
            sharded_step(shard, st, st["s"], y[a:b], g)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), f=st["f"].numpy(), s=st["s"].numpy(), D=st["D"],
                 g=g.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("T", [4, 5])
def test_gloo_two_ranks_match_unsharded_oracle(T, tmp_path):
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mp.start_processes(_rank, args=(2, port, T, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0, r1 = (np.load(tmp_path / f"rank{r}.npz") for r in range(2))
    # the update is deterministic: both ranks hold the same state
    assert np.array_equal(r0["f"], r1["f"]) and np.array_equal(r0["s"], r1["s"])
    # and it equals the unsharded oracle: two steps over all transmitters
    from oracle import fista, grad
    from paper_1708_01663_gb300 import synth
    n, angles, rx, prob = _problem(T)
    f_true = synth.ellipse_phantom(n, 2, (0.1, 0.4), 3)
    _, y, _, _ = grad.forward(prob, f_true, tol=1e-12)
    ref, hist = fista.relaxed_fista(prob, y, 0.5 * f_true, 0.5, 1e-3, 0.96, 2, 10, box_re=(-np.inf, np.inf),
                                    tol=1e-12)
    assert abs(float(r0["D"]) - hist[-1]) <= 1e-9 * hist[-1]
    assert np.linalg.norm(r0["f"] - ref) <= 1e-9 * np.linalg.norm(ref)
