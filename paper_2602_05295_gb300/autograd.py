"""torch.autograd.Function over the checkpointed forward and the discrete adjoint.

``MELBMFunction.apply(u0, F, sim, nsteps, K)`` runs ``nsteps`` FP32-storage steps
from the initial state (rho = 1, u = u0, S = u0 u0) with the body force F, keeping
a 16-bit checkpoint every K steps (every FP32 state when nsteps <= K, so that the
backward pass needs no recompute), and returns the final public moments as a
(10, N) tensor (rho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz).  Its backward
calls melbm_backward: the hand-written adjoint kernels return dL/du0 and dL/dF.
All arithmetic runs in the CUDA library; this module only passes tensors.
"""
from __future__ import annotations

import torch


class MELBMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, F, sim, nsteps, K):
        u0 = u0.detach().to(torch.float32).contiguous()
        F = F.detach().to(torch.float32).contiguous()
        sim.set_force(F)
        sim.forward_checkpointed(u0, nsteps, K)
        rho, u, S = sim.get_moments()
        ctx.sim = sim
        return torch.cat([rho[None], u, S], 0)

    @staticmethod
    def backward(ctx, grad_out):
        sim = ctx.sim
        N = sim.N
        g_u0 = torch.empty(3, N, dtype=torch.float32, device=grad_out.device)
        g_F = torch.empty(3, N, dtype=torch.float32, device=grad_out.device)
        sim.backward(grad_out.to(torch.float32).contiguous(), g_u0, g_F)
        return g_u0, g_F, None, None, None


def kinetic_energy_in_region(m, region_mask):
    """L = sum over the region of rho |u|^2 / 2 from public moments (10, N)."""
    rho, u = m[0], m[1:4]
    return 0.5 * (rho * (u * u).sum(0))[region_mask].sum()
