"""Differentiable propagation: a torch.autograd.Function over the C ABI.

forward  y = A x  (cwo_propagate_batch: pad, FFT, H, inverse FFT, crop)
backward grad_x = A^H grad_y  (cwo_propagate_adjoint_batch: the same passes with conj(H))

A is complex-linear, so with PyTorch's conjugate-Wirtinger convention the vector-Jacobian product
is exactly the adjoint map; it is computed by the hand-written adjoint kernels, not by autograd
tracing through FFTs.
"""
from __future__ import annotations

import torch

from . import cwo


class _Propagate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, plan: cwo.Plan, z):
        ctx.plan = plan
        ctx.z = z
        xb = x.reshape(-1, plan.ny, plan.nx).contiguous()
        y = plan.propagate_batch(xb, z=z)
        return y.reshape(x.shape)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        plan = ctx.plan
        gb = g.reshape(-1, plan.ny, plan.nx).contiguous()
        gx = plan.propagate_batch(gb, z=ctx.z, adjoint=True)
        return gx.reshape(g.shape), None, None


def propagate(x: torch.Tensor, plan: cwo.Plan, z=None) -> torch.Tensor:
    """Differentiable propagation of complex64 fields [..., Ny, Nx] with ``plan``.

    ``z``: None (the plan's distance) or a sequence with one distance per field."""
    if x.dtype != torch.complex64:
        raise TypeError("propagate expects complex64 fields")
    return _Propagate.apply(x, plan, None if z is None else list(z))
