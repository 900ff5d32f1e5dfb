"""``torch.autograd.Function`` around the fused loss + adjoint of the C ABI.

The forward pass calls ``ptycho_adjoint`` when a gradient is required: the library
evaluates the loss and the analytic gradient (the reverse pass of Fig. 1B) in one fused
sweep, recomputing or keeping its FFT fields internally, so no per-position intermediate
is stored on the autograd tape; only the two parameter-sized gradients are kept for
``backward``.  Without a gradient requirement it calls ``ptycho_loss``.
"""
from __future__ import annotations

import torch

from .api import Plan


class PtychoLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, O, P, plan: Plan, Imeas, sigma=None, bg=None, mask=None, batch=None):
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            loss, gO, gP = plan.adjoint(O.detach(), P.detach(), Imeas, sigma, bg, mask, batch)
            ctx.save_for_backward(gO, gP)
        else:
            loss = plan.loss(O.detach(), P.detach(), Imeas, sigma, bg, mask, batch)
        return loss.reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        gO, gP = ctx.saved_tensors
        s = grad_out.to(torch.float32)
        return gO * s, gP * s, None, None, None, None, None, None


def ptycho_loss(O, P, plan: Plan, Imeas, sigma=None, bg=None, mask=None, batch=None):
    """Differentiable FP64 loss of complex64 parameters O (packed) and P ([L, M, F, F])."""
    return PtychoLoss.apply(O, P, plan, Imeas, sigma, bg, mask, batch)
