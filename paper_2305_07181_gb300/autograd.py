"""torch.autograd.Function over the library's residual and its reverse mode.

    r = residual(u, solver)      # forward: esplit_residual
    r.backward(cot)              # backward: esplit_residual_vjp

Both directions run in the CUDA library; this module only routes tensors.
"""
from __future__ import annotations

import torch


class ResidualFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u: torch.Tensor, solver):
        u = u.contiguous()
        ctx.solver = solver
        ctx.save_for_backward(u)
        return solver.residual(u)

    @staticmethod
    def backward(ctx, cot: torch.Tensor):
        (u,) = ctx.saved_tensors
        grad = ctx.solver.residual_vjp(u, cot.contiguous())
        return grad, None


def residual(u: torch.Tensor, solver) -> torch.Tensor:
    """du/dt of the solver's scheme, differentiable through the library's VJP."""
    return ResidualFunction.apply(u, solver)
