"""torch.autograd.Function over the library's forward model and its
hand-written adjoint (Eqs. 1, 5, 6).

    model = spectrum_model(interp, theta, b)      # N x n_pix
    loss = f(model); loss.backward()              # theta.grad, b.grad

theta: N x 5 physical parameters (Teff, log g, [Fe/H], RV, sigma_v), b: N x
(D+1) Legendre continuum coefficients; both float32 CUDA tensors.  The
backward pass is lasp_backward (no generic autograd through the model).
"""
from __future__ import annotations

import torch


class SpectrumModel(torch.autograd.Function):
    @staticmethod
    def forward(ctx, interp, theta, b):
        theta = theta.contiguous()
        b = b.contiguous()
        ctx.interp = interp
        ctx.save_for_backward(theta, b)
        return interp.forward(theta, b)

    @staticmethod
    def backward(ctx, gmodel):
        theta, b = ctx.saved_tensors
        gth, gb = ctx.interp.backward(theta, b, gmodel.contiguous().to(torch.float32))
        return None, gth if ctx.needs_input_grad[1] else None, gb if ctx.needs_input_grad[2] else None


def spectrum_model(interp, theta, b):
    return SpectrumModel.apply(interp, theta, b)
