"""The Cox negative log partial likelihood as a torch.autograd.Function.

forward(beta) returns f(beta) = -(1/n) log partial likelihood (arXiv
2010.16114, Section 5.3, with the Section 6 Breslow ties) for each row of
beta (shape (k, p) or (p,)).  The backward pass is the gradient the solver
itself uses: the library's loss-and-gradient call runs the same two
genotype products and FP64 risk-set scans as one proximal-gradient step,
without the soft-threshold epilogue.  forward computes f and grad f in one
call and keeps grad f for backward.
"""
from __future__ import annotations

import torch

from .cox import CoxProblem


class CoxNLL(torch.autograd.Function):
    @staticmethod
    def forward(ctx, beta: torch.Tensor, problem: CoxProblem):
        loss, grad = problem.loss_grad(beta.detach().contiguous())
        ctx.save_for_backward(grad)
        ctx.vector = beta.dim() == 1
        out = torch.as_tensor(loss, dtype=torch.float64, device=beta.device)
        return out[0] if ctx.vector else out

    @staticmethod
    def backward(ctx, g_out):
        (grad,) = ctx.saved_tensors
        g_out = g_out.to(grad.dtype)
        if ctx.vector:
            return g_out * grad, None
        return g_out[:, None] * grad, None


def cox_nll(beta: torch.Tensor, problem: CoxProblem) -> torch.Tensor:
    """Differentiable f(beta) (one value per row of beta)."""
    return CoxNLL.apply(beta, problem)
