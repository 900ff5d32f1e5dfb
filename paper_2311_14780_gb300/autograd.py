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
        need = ctx.needs_input_grad
        sb = (len(need) > 4 and need[4]) or (len(need) > 5 and need[5])
        s_d = None if sigma is None else sigma.detach()
        b_d = None if bg is None else bg.detach()
        if sb:
            loss, gO, gP, gs, gb, _, _ = plan.adjoint_ex(O.detach(), P.detach(), Imeas, s_d, b_d, mask, batch,
                                                         want_z=False)
            ctx.save_for_backward(gO, gP, gs.reshape(sigma.shape) if sigma is not None else gs,
                                  gb.reshape(bg.shape) if bg is not None else gb)
        elif need[0] or need[1]:
            loss, gO, gP = plan.adjoint(O.detach(), P.detach(), Imeas, s_d, b_d, mask, batch)
            ctx.save_for_backward(gO, gP)
        else:
            loss = plan.loss(O.detach(), P.detach(), Imeas, s_d, b_d, mask, batch)
        return loss.reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        saved = ctx.saved_tensors
        s = grad_out.to(torch.float32)
        gO, gP = saved[0] * s, saved[1] * s
        gs = gb = None
        if len(saved) == 4:
            gs = saved[2] * s if ctx.needs_input_grad[4] else None
            gb = saved[3] * s if ctx.needs_input_grad[5] else None
        return gO, gP, None, None, gs, gb, None, None


def ptycho_loss(O, P, plan: Plan, Imeas, sigma=None, bg=None, mask=None, batch=None):
    """Differentiable FP64 loss of complex64 parameters O (packed) and P ([L, M, F, F]),
    and of the power coefficients sigma ([J]) and background bg ([F, F]) when they require
    a gradient."""
    return PtychoLoss.apply(O, P, plan, Imeas, sigma, bg, mask, batch)
