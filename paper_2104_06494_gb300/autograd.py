"""Differentiable integrals: PAGANI's estimate as a torch.autograd.Function.

Forward runs the adaptive integration (pagani_integrate_ex with
keep_leaves=1) and keeps the converged leaf set, the boxes whose rule values
sum to the estimate, as CUDA tensors.  Backward evaluates d/dtheta of the
rule estimate over that frozen leaf set with one kernel (pagani_gradient):
sum over boxes of vol sum_points w df/dtheta, for the positive product
families (product peak, Gaussian, C0), whose integrand is a product of
per-axis factors.  The leaf set is checkpointed once per forward instead of
keeping per-iteration region lists.
"""
from __future__ import annotations

import torch

from . import pagani_gradient, pagani_integrate_ex, pagani_leaves


class PaganiIntegral(torch.autograd.Function):
    """I(theta) = integral over [0,1]^dim of f(x; theta); theta is the
    family's parameter vector (float64 tensor, layout of include/pagani.h)."""

    @staticmethod
    def forward(ctx, theta, dim: int, family: int, epsrel: float, epsabs: float = 1e-20,
                max_regions: int = 10_000_000):
        params = theta.detach().cpu().double().numpy()
        r = pagani_integrate_ex(dim, family, params, epsrel, epsabs, max_regions, keep_leaves=1)
        if r.n_leaves < 0:
            raise RuntimeError("the leaf set was not kept (leaf log full)")
        lower, level = pagani_leaves(dim)
        ctx.save_for_backward(theta.detach())
        ctx.leaves = (lower, level)
        ctx.meta = (dim, family)
        ctx.result = r
        return theta.new_tensor(r.estimate)

    @staticmethod
    def backward(ctx, grad_out):
        (theta,) = ctx.saved_tensors
        dim, family = ctx.meta
        lower, level = ctx.leaves
        _, g = pagani_gradient(dim, family, theta.cpu().double().numpy(), lower, level)
        grad = torch.as_tensor(g, dtype=theta.dtype, device=theta.device) * grad_out
        return grad, None, None, None, None, None


def integral(theta, dim: int, family: int, epsrel: float, epsabs: float = 1e-20, max_regions: int = 10_000_000):
    return PaganiIntegral.apply(theta, dim, family, epsrel, epsabs, max_regions)
