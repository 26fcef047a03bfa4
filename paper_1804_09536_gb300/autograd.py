"""torch.autograd.Function for the spectral-weight loss of config "512^3 loss + gradient".

loss(x) = sum_k |F(x)_k w_k|^2, F the plan's forward transform (stage 0 ->
stage g, paper normalisation).  Backward: d loss / d x = 2 F^H (w^2 F x)
(d/dRe + i d/dIm convention used by torch for complex inputs), computed as
the gradient seed z = 2 g w^2 y followed by the adjoint transform
(tfft_adjoint: the backward passes with the redistributions reversed and
1/N).  Every step runs in the library's kernels; the forward output y is
kept for the backward.
"""
from __future__ import annotations

import torch


class SpectralWeightLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, w: torch.Tensor, plan) -> torch.Tensor:
        y = plan.forward(x)                        # keeps x (workspace)
        loss = plan.weighted_energy(plan.g, y, w)  # float64, deterministic
        ctx.save_for_backward(y, w)
        ctx.plan = plan
        return loss

    @staticmethod
    def backward(ctx, gout: torch.Tensor):
        y, w = ctx.saved_tensors
        plan = ctx.plan
        g = gout.detach().to(torch.float64).reshape(()).contiguous()
        z = plan.weight_scale(plan.g, y, w, g, 2.0)   # 2 g w^2 y
        gx = plan.adjoint(z)
        return gx, None, None


def spectral_weight_loss(x: torch.Tensor, w: torch.Tensor, plan) -> torch.Tensor:
    """sum |F(x) w|^2 with a gradient through the adjoint transform."""
    return SpectralWeightLoss.apply(x, w, plan)
