"""torch.autograd view of the SP2 density: forward is Eq. DM0, backward is the
adjoint (backward susceptibility) recursion of Eq. DM2.

For a scalar loss l(D), backward receives G = dl/dD and returns
dl/dH = chi^G, the susceptibility of the "observable" G (Eq. Suscept with
A = G). X_n is kept every ``ckpt_k`` steps during the forward pass and the
other X_n are recomputed segment by segment in backward (Sec. IV.A notes that
Eq. DM2 needs the X_n sequence stored).

H is symmetric by assumption (Sec. I), so only the symmetric part of G pairs
with admissible perturbations of H; backward uses (G + G^T)/2 and returns a
symmetric gradient: the gradient with respect to symmetric perturbations.
"""
from __future__ import annotations

import torch

from .api import Handle, sp2_adjoint, sp2_density


class SP2Density(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, nocc, mode, ckpt_k, handle):
        h = handle if handle is not None else Handle()
        D, info = sp2_density(H.detach().contiguous(), nocc, mode=mode, handle=h,
                              keep_history=True, ckpt_k=ckpt_k)
        ctx.handle = h
        ctx.info = info
        return D

    @staticmethod
    def backward(ctx, G):
        grad = sp2_adjoint(G.contiguous(), ctx.handle)
        return grad, None, None, None, None


def sp2_density_autograd(H: torch.Tensor, nocc: float, mode: str = "bf16x2", ckpt_k: int = 4,
                         handle: Handle | None = None) -> torch.Tensor:
    """Differentiable D(H). One handle holds one kept history: pass distinct
    handles (or none) for densities that are alive at the same time."""
    return SP2Density.apply(H, nocc, mode, ckpt_k, handle)
