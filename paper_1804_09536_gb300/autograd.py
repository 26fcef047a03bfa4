"""torch.autograd.Function for the spectral-weight loss of config "512^3 loss + gradient".

loss(x) = sum_k |F(x)_k w_k|^2, F the plan's forward transform (stage 0 ->
stage g, paper normalisation).  Backward: d loss / d x = 2 F^H (w^2 F x)
(d/dRe + i d/dIm convention used by torch for complex inputs).  The forward
sweep that sums the loss also writes u = w^2 y over y (one pass over y and w);
the backward is tfft_weighted_energy_grad: the adjoint transform of u (the
backward passes with the redistributions reversed and 1/N) whose last pass
also applies the factor 2 and the upstream gradient g, read on the device, so
the gradient seed is never materialised.  Every step, the factor 2 included,
runs in the library's kernels; torch only hands over g's device pointer.
"""
from __future__ import annotations

import torch


class SpectralWeightLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, w: torch.Tensor, plan) -> torch.Tensor:
        y = plan.forward(x)                             # keeps x (workspace)
        loss = plan.weighted_energy(plan.g, y, w, u=y)  # float64, deterministic; y <- w^2 y
        ctx.save_for_backward(y)
        ctx.plan = plan
        return loss

    @staticmethod
    def backward(ctx, gout: torch.Tensor):
        (u,) = ctx.saved_tensors
        plan = ctx.plan
        if gout.dtype != torch.float64:
            raise TypeError("the loss is float64, so is its upstream gradient")
        g = gout.detach().reshape(()).contiguous()  # a view of the same device scalar
        gx = plan.weighted_energy_grad(u, g)  # 2 g F^H (w^2 y); u kept (a retained graph may run it again)
        return gx, None, None


def spectral_weight_loss(x: torch.Tensor, w: torch.Tensor, plan) -> torch.Tensor:
    """sum |F(x) w|^2 with a gradient through the adjoint transform."""
    return SpectralWeightLoss.apply(x, w, plan)
