"""torch.autograd.Function wrappers of the drift product and the Chebyshev
Brownian term, differentiable with respect to bead positions R, forces F and
Wiener increments dW.

Forward and backward both run in libbdgb (bd_build_D, bd_apply_D,
bd_chebyshev_sqrt, bd_apply_D_backward, bd_chebyshev_backward); this module
only marshals tensors.  The backward rebuilds D(R) from the saved positions
(the caller's D buffer may have been reused since the forward) and recomputes
each pair's derivative instead of storing dD/dR.  Eigenvalue bounds and N_Ch
are treated as constants (no derivative through them).
"""
from __future__ import annotations

import torch

from . import binding


class BDSystem:
    """A plan plus a D buffer for autograd use (one system, one precision)."""

    def __init__(self, params: dict, precision: str = "fp64", max_rhs: int = 1,
                 max_cheb: int = 64):
        self.plan = binding.Plan(params, precision, max_rhs=max_rhs, max_cheb=max_cheb)
        self.D = self.plan.alloc_D()

    def build(self, R: torch.Tensor):
        self.plan.build_D(R.detach().contiguous(), self.D)


class DApply(torch.autograd.Function):
    """Y = D(R) F  (Eq. sde drift product; Y and F are 3N vectors)."""

    @staticmethod
    def forward(ctx, R, F, system: BDSystem):
        R = R.detach().contiguous()
        F = F.detach().contiguous()
        system.build(R)
        Y = torch.empty_like(F)
        system.plan.apply(system.D, F.view(1, -1), Y.view(1, -1),
                          refine=system.plan.precision != "fp64")
        ctx.system = system
        ctx.save_for_backward(R, F)
        return Y

    @staticmethod
    def backward(ctx, gY):
        R, F = ctx.saved_tensors
        system = ctx.system
        system.build(R)
        gY = gY.contiguous()
        gR = torch.empty(R.numel(), dtype=torch.float64, device=R.device)
        gF = torch.empty_like(F) if ctx.needs_input_grad[1] else None
        system.plan.apply_backward(R, system.D, F, gY, gR, gF)
        return gR.view_as(R), gF, None


class ChebSqrt(torch.autograd.Function):
    """dS = P(D(R)) dW, Fixman's Chebyshev series (Eqs. cheb1-cheb3);
    dW and dS are (m, 3N); bounds is a device tensor {d_min, d_max}."""

    @staticmethod
    def forward(ctx, R, dW, bounds, n_cheb: int, system: BDSystem):
        R = R.detach().contiguous()
        dW = dW.detach().contiguous()
        system.build(R)
        dS = torch.empty_like(dW)
        system.plan.chebyshev(system.D, bounds, n_cheb, dW, dS)
        ctx.system, ctx.n_cheb = system, n_cheb
        ctx.save_for_backward(R, dW, bounds)
        return dS

    @staticmethod
    def backward(ctx, gS):
        R, dW, bounds = ctx.saved_tensors
        system = ctx.system
        system.build(R)
        gR = torch.empty(R.numel(), dtype=torch.float64, device=R.device)
        gdW = torch.empty_like(dW) if ctx.needs_input_grad[1] else None
        system.plan.chebyshev_backward(R, system.D, bounds, ctx.n_cheb, dW, gS.contiguous(),
                                       gR, gdW)
        return gR.view_as(R), gdW, None, None, None


def drift(R, F, system: BDSystem):
    return DApply.apply(R, F, system)


def brownian(R, dW, bounds, n_cheb, system: BDSystem):
    return ChebSqrt.apply(R, dW, bounds, n_cheb, system)
