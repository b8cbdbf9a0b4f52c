"""torch.autograd wrapper: effective tensor as a differentiable function of a
per-voxel stiffness scale field.

For A_beta = s_beta A_phase(beta), the discrete effective tensor satisfies
e_i.A*_h e_j = A0_ij + h^d b_i^T K^{-1} b_j with K the symmetric operator of
Eq. (13), whose local part M_beta = (s_beta A_phase - A0)^{-1} is the only
term that depends on s.  Differentiating, with tau_j = K^{-1} b_j and
eps_j = M tau_j (the strain estimate of Table 1's second criterion):

    d(e_i.A*_h e_j)/d s_beta = h^d eps_i,beta . A_phase(beta) eps_j,beta.

Because K is self-adjoint, the adjoint solutions are the forward
polarisations: backward needs no extra solve and no stored CG iterates, only
the c polarisations kept from the forward pass (c * c * V doubles).  The
gradient contraction runs in the CUDA library (lsh_effective_grad).
"""
from __future__ import annotations

import numpy as np
import torch

from . import lsh


class EffectiveTensor(torch.autograd.Function):
    """A*_h(s) (c x c, float64) for a handle built with a scale field."""

    @staticmethod
    def forward(ctx, scale: torch.Tensor, handle: "lsh.Handle", tol: float = 1e-10, maxit: int = 10000):
        handle.set_microstructure(handle.phase_source, scale.detach().float().contiguous())
        A, infos, tau = handle.effective(tol=tol, maxit=maxit, return_tau=True)
        ctx.handle = handle
        ctx.scale_dtype = scale.dtype
        ctx.save_for_backward(tau)
        ctx.infos = infos
        return torch.from_numpy(A).to(device=scale.device)

    @staticmethod
    def backward(ctx, grad_A: torch.Tensor):
        (tau,) = ctx.saved_tensors
        W = np.ascontiguousarray(grad_A.detach().to(torch.float64).cpu().numpy())
        g = ctx.handle.effective_grad(tau, W)
        return g.to(ctx.scale_dtype), None, None, None


def effective_tensor(scale: torch.Tensor, handle: "lsh.Handle", tol: float = 1e-10, maxit: int = 10000):
    """Differentiable A*_h with respect to the per-voxel scale field."""
    return EffectiveTensor.apply(scale, handle, tol, maxit)
