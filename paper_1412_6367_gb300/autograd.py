"""Differentiable azimuthal integration: torch.autograd.Function over the CUDA forward and
its hand-written adjoint kernel (gather over the pixel-major matrix)."""
from __future__ import annotations

import torch

from .api import Integrator


class AzimuthalIntegrate(torch.autograd.Function):
    """I = integrate(image, flat) with gradients for the image and the flat field.

    forward(image, flat, integrator, dark=None, solid_angle=None, polarization=None,
            precision="fp32") -> I
    The image may be float32 / int32 / uint32; its gradient is returned in the
    accumulation dtype (float64 for "fp64", float32 for "fp32").  The gradient for the dark
    current is minus the image gradient.
    """

    @staticmethod
    def forward(ctx, image, flat, integrator: Integrator, dark=None, solid_angle=None,
                polarization=None, precision="fp32"):
        res = integrator.integrate(image, dark, flat, solid_angle, polarization, precision)
        ctx.integrator = integrator
        ctx.precision = precision
        ctx.flat_given = flat is not None
        ctx.image_dtype = image.dtype if image.is_floating_point() else res.I.dtype
        ctx.flat_dtype = flat.dtype if flat is not None else res.I.dtype
        ctx.save_for_backward(res.I.reshape(-1), res.sum_norm.reshape(-1), solid_angle, polarization)
        return res.I

    @staticmethod
    def backward(ctx, grad_I):
        I, N, sa, pol = ctx.saved_tensors
        dt = I.dtype
        g = grad_I.reshape(-1).to(dt).contiguous()
        want_img = ctx.needs_input_grad[0]
        want_flat = ctx.needs_input_grad[1] and ctx.flat_given
        gi, gf = ctx.integrator.backward(g, I, N, sa, pol, ctx.precision, want_image=want_img,
                                         want_flat=want_flat)
        if gi is not None:
            gi = gi.to(ctx.image_dtype)
        if gf is not None:
            gf = gf.to(ctx.flat_dtype)
        return gi, gf, None, None, None, None, None


def integrate(image, flat, integrator, dark=None, solid_angle=None, polarization=None,
              precision="fp32"):
    return AzimuthalIntegrate.apply(image, flat, integrator, dark, solid_angle, polarization,
                                    precision)
