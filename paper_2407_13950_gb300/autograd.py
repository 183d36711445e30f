"""torch.autograd.Function over the hand-written adjoint kernel.

``ms_objective(problem, alpha, W)`` returns the multiple-shooting objective P as a 0-d float64
tensor on the problem's device.  When alpha or W requires grad, the forward call runs the full
evaluation (forward sweep + discrete adjoint sweep, one library call) and keeps dP/dalpha and
dP/dW; backward scales them by the incoming gradient.  Otherwise only the objective is
evaluated.  alpha and W must be contiguous float64 CUDA tensors.
"""
from __future__ import annotations

import torch

from .msqoc import Problem


class MSObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alpha: torch.Tensor, W: torch.Tensor, problem: Problem):
        if alpha.device.type != "cuda" or alpha.dtype != torch.float64:
            raise TypeError("alpha must be a float64 CUDA tensor")
        alpha = alpha.contiguous()
        M = problem.spec.M
        if M > 1:
            if W.device != alpha.device or W.dtype != torch.float64:
                raise TypeError("W must be a float64 tensor on alpha's device")
            W = W.contiguous()
        stream = torch.cuda.current_stream(alpha.device)
        P = torch.zeros((), dtype=torch.float64, device=alpha.device)
        need = ctx.needs_input_grad[0] or (M > 1 and ctx.needs_input_grad[1])
        if need:
            ga = torch.empty(problem.d, dtype=torch.float64, device=alpha.device)
            gW = torch.empty(max(problem.nW, 1), dtype=torch.float64, device=alpha.device)
            problem.eval_gradient_into(alpha, W if M > 1 else None, P, ga, gW if M > 1 else None, stream=stream)
            ctx.save_for_backward(ga, gW[:problem.nW])
        else:
            problem.eval_objective_into(alpha, W if M > 1 else None, P, stream=stream)
        ctx.M = M
        return P

    @staticmethod
    def backward(ctx, gP: torch.Tensor):
        ga, gW = ctx.saved_tensors
        dW = gP * gW if ctx.M > 1 else None
        return gP * ga, dW, None


def ms_objective(problem: Problem, alpha: torch.Tensor, W: torch.Tensor) -> torch.Tensor:
    return MSObjective.apply(alpha, W, problem)
