"""torch.autograd view of the SPECT system matrix and the Poisson likelihood.

``SpectProjector.apply(x, plan, subset)`` is H x (Eq. 1 of PyTomography,
arXiv 2309.01977) for a volume or a batch of volumes; its backward is the
library's exact transpose H^T (``spect_back``).  H is linear, so nothing but
the plan is kept for the backward pass: every angle's rotation is recomputed
there instead of storing rotated volumes.

``PoissonLogLikelihood.apply(p, y, s, plan)`` is L = sum y log(p + s) - (p + s)
(Table 1, log y! dropped) with the gradient y / (p + s) - 1 computed by the
same kernel.  Chained, autograd gives the Poisson gradient of Table 1,
grad_x L = H^T(y / (Hx + s)) - H^T 1.
"""
from __future__ import annotations

import torch

from . import spect


class SpectProjector(torch.autograd.Function):
    """proj = H_subset x; x is [n][n][nz] or [batch][n][n][nz] (CUDA float32)."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, plan: "spect.Plan", subset: int = -1):
        ctx.plan = plan
        ctx.subset = subset
        ctx.x_shape = x.shape
        return plan.forward(x.contiguous(), subset)

    @staticmethod
    def backward(ctx, grad_proj: torch.Tensor):
        g = ctx.plan.back(grad_proj.contiguous(), ctx.subset)
        return g.reshape(ctx.x_shape), None, None


class PoissonLogLikelihood(torch.autograd.Function):
    """L = sum y log(p + s) - (p + s) as a float64 scalar; dL/dp = y/(p+s) - 1."""

    @staticmethod
    def forward(ctx, p: torch.Tensor, y: torch.Tensor, s: float, plan: "spect.Plan"):
        p = p.contiguous()
        y = y.contiguous()
        ll, grad = plan.poisson_ll(y, p, s, grad=True)
        ctx.save_for_backward(grad)
        return ll[0]

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        (grad,) = ctx.saved_tensors
        return grad * g.to(grad.dtype), None, None, None


def poisson_loss(x: torch.Tensor, y: torch.Tensor, s: float, plan: "spect.Plan", subset: int = -1):
    """Poisson log-likelihood of volume(s) x against counts y (differentiable in x)."""
    return PoissonLogLikelihood.apply(SpectProjector.apply(x, plan, subset), y, s, plan)
