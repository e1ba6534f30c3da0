"""Differentiable dose operator and thresholded loss (torch.autograd over the C ABI).

DoseFn.apply(proj, projector) -> dose = A proj (vamrt_forward_dose).  Its backward is
the projection kernel: dL/dproj = A^T dL/ddose (vamrt_adjoint), recomputing every ray
path per call instead of storing paths.  ThresholdLossFn.apply(dose, target, d_l, d_h)
-> L (vamrt_threshold_loss), whose gradient is produced by the same call.
"""
from __future__ import annotations

import torch

from . import vamrt


class DoseFn(torch.autograd.Function):
    """dose = A proj.  With storage_dtype = bfloat16 the projections handed to the kernel
    (and the dose it writes) are stored in BF16 while every sum runs in FP32; the
    gradient with respect to the (FP32) projections stays FP32."""

    @staticmethod
    def forward(ctx, proj: torch.Tensor, projector: "vamrt.Projector", storage_dtype=None):
        storage = storage_dtype or proj.dtype
        ctx.projector = projector
        ctx.proj_dtype = proj.dtype
        stored = proj.detach().to(storage).contiguous()
        return projector.forward_dose(stored, dose_dtype=storage)

    @staticmethod
    def backward(ctx, grad_dose: torch.Tensor):
        gd = grad_dose.contiguous()
        if gd.dtype not in (torch.float32, torch.bfloat16):
            gd = gd.float()
        grad_proj = ctx.projector.adjoint(gd, proj_dtype=torch.float32)
        return grad_proj.to(ctx.proj_dtype), None, None


class ThresholdLossFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, dose: torch.Tensor, target: torch.Tensor, projector: "vamrt.Projector", d_l: float,
                d_h: float):
        loss, grad = projector.threshold_loss(dose.contiguous(), target, d_l, d_h, grad=True)
        ctx.save_for_backward(grad)
        ctx.dose_dtype = dose.dtype
        return loss

    @staticmethod
    def backward(ctx, grad_loss: torch.Tensor):
        (grad,) = ctx.saved_tensors
        return (grad * grad_loss.to(grad.dtype)).to(ctx.dose_dtype), None, None, None, None


def dose(proj: torch.Tensor, projector: "vamrt.Projector", storage_dtype=None) -> torch.Tensor:
    return DoseFn.apply(proj, projector, storage_dtype)


def threshold_loss(dose_vol: torch.Tensor, target: torch.Tensor, projector: "vamrt.Projector", d_l: float = 0.9,
                   d_h: float = 1.0) -> torch.Tensor:
    return ThresholdLossFn.apply(dose_vol, target, projector, d_l, d_h)
