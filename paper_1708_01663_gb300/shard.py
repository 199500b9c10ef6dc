"""Transmitter sharding of a relaxed-FISTA step.

D (Eq. 7) and the gradient vector g of Prop. 1 are sums over transmitters,
and every transmitter's forward and adjoint solves (Eq. 13) are independent.
So the transmitters split into contiguous blocks, one per rank: each rank
holds f, the Green spectrum and H, and builds a context for its own block of
transmitters only.  A step is then

    (D_r, g_r) = cisor_grad on the rank's transmitters      (no communication)
    (D, g)     = sum over ranks                            (one all-reduce)
    f_k, s_{k+1}, t_{k+1} = cisor_step_update(g, D)        (Eqs. 9-11, redundant)

The update is deterministic, so every rank ends with the same state and no
broadcast is needed.  The all-reduce uses whatever backend the process group
has (NCCL for device tensors, gloo for host tensors).
"""
from __future__ import annotations


def tx_split(T: int, world: int, rank: int) -> tuple[int, int]:
    """[start, stop) of rank's transmitters: contiguous blocks whose sizes differ by at most one."""
    if not (0 <= rank < world) or T < world:
        raise ValueError(f"cannot split {T} transmitters over {world} ranks (rank {rank})")
    base, rem = divmod(T, world)
    start = rank * base + min(rank, rem)
    return start, start + base + (1 if rank < rem else 0)


def allreduce_grad(g, D: float, group=None) -> float:
    """Sum the complex gradient tensor g in place and the scalar D over the ranks of ``group``;
    returns the summed D."""
    import torch
    import torch.distributed as dist
    dist.all_reduce(torch.view_as_real(g), group=group)
    d = torch.tensor([float(D)], dtype=torch.float64, device=g.device)
    dist.all_reduce(d, group=group)
    return float(d.item())


def sharded_step(ctx, state, s, y_local, g, reduce=allreduce_grad, tol=1e-4, max_iter=2000, x0_mode=2,
                 check=True):
    """One relaxed-FISTA step with this rank's transmitters.

    ctx: the rank's Cisor context (its transmitters only); state: its
    FistaState, whose s points at the tensor ``s``; y_local: the measurements
    of its transmitters [T_r, M]; g: an [N] complex64 device tensor that
    receives the summed gradient.  Returns (status, solve info) of the
    rank's gradient."""
    D, st, info = ctx.grad(s, y_local, g, tol=tol, max_iter=max_iter, x0_mode=x0_mode, check=check)
    D = reduce(g, D)
    ctx.step_update(state, g, D)
    return st, info
