"""torch.autograd.Function for the fermionic action S_F(x) (Sec. II D).

    S_F(x; Phi) = (1/2) sum_sigma Phi_sigma^T (A^T A)^{-1} Phi_sigma,  A = M(x) Lambda(x)

at fixed pseudofermions Phi (Eq. (S_F)). Forward: hol_set_field(x),
b = Lambda^{-T} Phi (phi_to_rhs), v = (M^T M)^{-1} b (cg_solve), S_F =
(1/2) sum b.v (Eq. (Sf_Psi), the action-only mode of the force call); only
x, v and b are kept. Backward: the hand-written adjoint kernel (the force
call, Eq. (dSF_dx)) at the saved field, which recomputes B_tau v_{tau-1}
slice by slice from v instead of storing any product of B matrices
(recompute rather than checkpoint). A forward whose result is never
differentiated pays for no force. Every step runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import HOL_F32, HOL_F64, Context


class FermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx_, x: torch.Tensor, Phi: torch.Tensor, lib_ctx: Context, tol: float,
                prec: int, precond: bool):
        xd = x.detach().contiguous()
        lib_ctx.set_field(xd)
        b = torch.empty_like(Phi)
        lib_ctx.phi_to_rhs(Phi.detach().contiguous(), b)
        v = torch.empty_like(Phi)
        lib_ctx.cg_solve(b, v, tol=tol, prec=prec, precond=precond)
        sf = torch.empty(1, dtype=torch.float64, device=x.device)
        lib_ctx.force(v, b, None, with_bosonic=False, S_F=sf)
        ctx_.lib_ctx = lib_ctx
        ctx_.save_for_backward(xd.clone(), v, b)
        return sf[0]

    @staticmethod
    def backward(ctx_, grad_out):
        x, v, b = ctx_.saved_tensors
        lib = ctx_.lib_ctx
        # the context may hold another field by now (e.g. a second forward)
        lib.set_field(x)
        F = torch.empty_like(x)
        lib.force(v, b, F, with_bosonic=False)
        return grad_out * F, None, None, None, None, None


def fermion_action(x: torch.Tensor, Phi: torch.Tensor, lib_ctx: Context, tol: float = 1e-10,
                   prec: int = HOL_F64, precond: bool = False) -> torch.Tensor:
    """S_F(x) as a differentiable scalar (FP64 tensor on the GPU)."""
    return FermionAction.apply(x, Phi, lib_ctx, tol, prec, precond)


__all__ = ["FermionAction", "fermion_action", "HOL_F32", "HOL_F64"]
