"""torch.autograd.Function for the fermionic action S_F(x) (Sec. II D).

    S_F(x; Phi) = (1/2) sum_sigma Phi_sigma^T (A^T A)^{-1} Phi_sigma,  A = M(x) Lambda(x)

at fixed pseudofermions Phi (Eq. (S_F)). Forward: hol_set_field(x),
b = Lambda^{-T} Phi (phi_to_rhs), v = (M^T M)^{-1} b (cg_solve), S_F =
(1/2) sum b.v (Eq. (Sf_Psi)). Backward: dS_F/dx from the hand-written force
kernel (Eq. (dSF_dx)), which recomputes B_tau v_{tau-1} slice by slice instead
of storing any product of B matrices; only v and b are kept between forward
and backward. Every step runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import HOL_F32, HOL_F64, Context


class FermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx_, x: torch.Tensor, Phi: torch.Tensor, lib_ctx: Context, tol: float,
                prec: int, precond: bool):
        lib_ctx.set_field(x.detach().contiguous())
        b = torch.empty_like(Phi)
        lib_ctx.phi_to_rhs(Phi.detach().contiguous(), b)
        v = torch.empty_like(Phi)
        lib_ctx.cg_solve(b, v, tol=tol, prec=prec, precond=precond)
        sf = torch.empty(1, dtype=torch.float64, device=x.device)
        F = torch.empty_like(x)
        # the force call also returns S_F = (1/2) sum b.v; keep F for backward
        lib_ctx.force(v, b, F, with_bosonic=False, S_F=sf)
        ctx_.save_for_backward(F)
        return sf[0]

    @staticmethod
    def backward(ctx_, grad_out):
        (F,) = ctx_.saved_tensors
        return grad_out * F, None, None, None, None, None


def fermion_action(x: torch.Tensor, Phi: torch.Tensor, lib_ctx: Context, tol: float = 1e-10,
                   prec: int = HOL_F64, precond: bool = False) -> torch.Tensor:
    """S_F(x) as a differentiable scalar (FP64 tensor on the GPU)."""
    return FermionAction.apply(x, Phi, lib_ctx, tol, prec, precond)


__all__ = ["FermionAction", "fermion_action", "HOL_F32", "HOL_F64"]
