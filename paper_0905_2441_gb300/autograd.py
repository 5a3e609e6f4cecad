"""torch.autograd.Function over the hand-written likelihood adjoint.

forward: l_p = smc_loglik_batch(theta) (the Section 4.1 mixture
log-likelihood per particle); backward: dL/dtheta = grad_output[p] *
d l_p / d mu_k, where the gradient comes from the same CUDA kernel run with
its fused adjoint (d l / d mu_k = sum_n r_nk (y_n - mu_k) / sigma^2).  The
scaling by grad_output is the one elementwise product torch performs.
"""
from __future__ import annotations

import torch

from . import api


class LogLikFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx_, theta: torch.Tensor, y: torch.Tensor, model: api.GMM, ctx: api.Context):
        theta = theta.contiguous()
        needs = theta.requires_grad
        grad = torch.empty_like(theta) if needs else None
        out = api.loglik_batch(ctx, model, y, theta.detach(), grad=grad)
        if needs:
            ctx_.save_for_backward(grad)
        return out

    @staticmethod
    def backward(ctx_, g_out: torch.Tensor):
        (grad,) = ctx_.saved_tensors
        return grad * g_out.to(grad.dtype)[None, :], None, None, None


def loglik(theta: torch.Tensor, y: torch.Tensor, model: api.GMM, ctx: api.Context):
    """Differentiable per-particle log-likelihood; theta is float32 [K][M]."""
    return LogLikFn.apply(theta, y, model, ctx)
