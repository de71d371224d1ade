"""Differentiable LBRS runs: torch.autograd.Function over the library's adjoint.

``run(U0, solver, n_steps)`` returns the conserved fields after n_steps
steps of a periodic D2Q4 problem started from f* = f^eq(U0).  Its backward
pass is the library's hand-written discrete adjoint with sqrt(T)
checkpointing (lbrs_forward_checkpointed / lbrs_backward_checkpointed): the
forward keeps the state every `segment` steps, the backward recomputes each
segment from its checkpoint while recording the moments and sweeps it with
the adjoint step.  The paper has no adjoint; this is the transpose of the
step it defines.
"""
from __future__ import annotations

import math

import torch


class LBRSRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0: torch.Tensor, solver, n_steps: int, segment: int):
        solver.set_state(U0.detach().contiguous(), primitive=False)
        solver.forward_checkpointed(n_steps, segment)
        ctx.solver = solver
        return solver.moments(dtype=U0.dtype)

    @staticmethod
    def backward(ctx, grad_UT: torch.Tensor):
        solver = ctx.solver
        gbar = solver.adjoint_seed(grad_UT.contiguous())
        grad = solver.backward_checkpointed(gbar)
        return grad.to(grad_UT.dtype), None, None, None


def run(U0: torch.Tensor, solver, n_steps: int, segment: int | None = None) -> torch.Tensor:
    """U(T) of n_steps LBRS steps from U0 (conserved fields, (4, ny, nx)), differentiable in U0."""
    return LBRSRun.apply(U0, solver, int(n_steps), int(segment or math.ceil(math.sqrt(n_steps))))
