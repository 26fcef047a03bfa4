"""torch.autograd.Function for the spectral-weight loss of config "512^3 loss + gradient".

loss(x) = sum_k |F(x)_k w_k|^2, F the plan's forward transform (stage 0 ->
stage g, paper normalisation).  Backward: d loss / d x = 2 F^H (w^2 F x)
(d/dRe + i d/dIm convention used by torch for complex inputs).  The forward
sweep that sums the loss also writes u = w^2 y over y (one pass over y and w);
the backward is the adjoint transform of u (tfft_adjoint: the backward passes
with the redistributions reversed and 1/N) with the factor 2 g applied on the
device by its last pass, so the gradient seed is never materialised.  Every
step runs in the library's kernels.
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
        c = (2.0 * gout.detach().to(torch.float64)).reshape(()).contiguous()
        gx = plan.adjoint(u, coef=c)  # 2 g F^H (w^2 y); u kept (a retained graph may run it again)
        return gx, None, None


def spectral_weight_loss(x: torch.Tensor, w: torch.Tensor, plan) -> torch.Tensor:
    """sum |F(x) w|^2 with a gradient through the adjoint transform."""
    return SpectralWeightLoss.apply(x, w, plan)
