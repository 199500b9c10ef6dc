"""D(f) of Eq. 7 as a torch.autograd.Function whose backward is the CUDA adjoint.

forward  -> cisor_data_term: field solves A u_t = u_in,t, residuals w_t and D;
            the fields u_t and w_t stay in the context's HBM as the checkpoint.
backward -> cisor_data_backward: the adjoint solves A^H v_t = diag(f)^H H^H w_t
            and g = sum_t conj(u_t)(H^H w_t + G^H v_t) (Prop. 1), scaled by the
            incoming gradient.
For a real f tensor the gradient is Re g; for a complex64 f it is
Re g + i Im g = dD/dRe f + i dD/dIm f, which is PyTorch's convention for the
gradient of a real loss with respect to a complex tensor.  One context holds
one pending backward: call backward before the next forward on that context.
"""
from __future__ import annotations

import torch


class DataTerm(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, y, cis, tol, max_iter):
        fc = (f if f.is_complex() else f.to(torch.complex64)).contiguous()
        D, _, info = cis.data_term(fc, y.contiguous(), tol=tol, max_iter=max_iter)
        ctx.cis, ctx.real, ctx.tol, ctx.max_iter, ctx.shape = cis, not f.is_complex(), tol, max_iter, f.shape
        ctx.fwd_info = info.as_dict()
        return torch.tensor(D, dtype=torch.float64, device=f.device)

    @staticmethod
    def backward(ctx, gD):
        g = torch.empty(ctx.shape, dtype=torch.complex64, device=gD.device)
        ctx.cis.data_backward(g, tol=ctx.tol, max_iter=ctx.max_iter)
        grad = g.real if ctx.real else g
        return grad * gD.to(grad.real.dtype), None, None, None, None


def data_term(f, y, cis, tol=1e-6, max_iter=3000):
    """D(f) = 1/2 sum_t ||H diag(u_t) f - y_t||^2 with a CUDA adjoint backward."""
    return DataTerm.apply(f, y, cis, tol, max_iter)
