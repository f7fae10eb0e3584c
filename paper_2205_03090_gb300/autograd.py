"""torch.autograd.Function over the flash: the forward pass is ptflash_flash,
the backward pass the implicit-function-theorem adjoint kernel
(ptflash_flash_adjoint).  Marshalling only: both passes run in the CUDA
library.  The feed z is read as mole numbers (results depend on z / sum z)."""
from __future__ import annotations

import torch

from . import ptflash


class FlashFunction(torch.autograd.Function):
    """(beta, x, y) = flash(P, T, z) for one fluid system (a ptflash.Flash)."""

    @staticmethod
    def forward(ctx, P, T, z, fl: ptflash.Flash):
        P, T, z = P.contiguous(), T.contiguous(), z.contiguous()
        out = fl.ptflash_flash(P, T, z)
        ctx.fl = fl
        ctx.res = out
        ctx.save_for_backward(P, T, z)
        ctx.mark_non_differentiable(out.nphase)
        return out.beta, out.x, out.y, out.nphase

    @staticmethod
    def backward(ctx, gbeta, gx, gy, _gnphase):
        P, T, z = ctx.saved_tensors
        gP, gT, gz, _ = ctx.fl.ptflash_flash_adjoint(P, T, z, ctx.res, gbeta, gx, gy)
        return gP, gT, gz, None


def flash(P, T, z, fl: ptflash.Flash):
    """Differentiable flash: returns beta[n], x[nc, n], y[nc, n], nphase[n]."""
    return FlashFunction.apply(P, T, z, fl)
