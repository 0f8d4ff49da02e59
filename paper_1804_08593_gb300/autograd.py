"""torch.autograd.Function for the pseudofermion action S = phi^dag (Mpc^dag Mpc)^-1 phi.

Forward: FP64 CG solve X = A^-1 phi and S = Re(2 phi^dag X - ||Mpc X||^2) (equal to
phi^dag A^-1 phi at the exact solution).  Backward: the gradient with respect to the links
from X alone — A is Hermitian, so the adjoint solve is the forward solve — and the fused
per-link outer-product force kernel (dwf_force).  Gradients use PyTorch's complex convention.
"""
from __future__ import annotations

import torch

from . import dwf


class PseudofermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, phi, handle, tol=1e-12, maxit=1000000):
        dwf.dwf_update_links(handle, U.detach().contiguous())
        phi_c = phi.detach().contiguous()
        X = torch.zeros_like(phi_c)
        dwf.dwf_cg(handle, phi_c, X, tol, maxit, "f64")
        S = dwf.dwf_action(handle, phi_c, X)
        ctx.save_for_backward(U.detach(), phi_c, X)
        ctx.handle = handle
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, gS):
        U, phi, X = ctx.saved_tensors
        dwf.dwf_update_links(ctx.handle, U.contiguous())
        dSdU = torch.empty_like(U)
        dwf.dwf_force(ctx.handle, phi, X, dSdU)
        return gS.to(dSdU.dtype) * dSdU, None, None, None, None


def pseudofermion_action(U, phi, handle, tol=1e-12):
    return PseudofermionAction.apply(U, phi, handle, tol)
