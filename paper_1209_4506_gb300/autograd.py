"""torch.autograd.Function wrappers of the Hartree energy (adjoint by the library's kernels).

HartreeEnergy(rho)      E_H of a density on the grid.  dE_H/drho_r = V_H(r) dV: the
                        Poisson operator is self-adjoint, so the backward pass is one
                        more solve of the same density (recomputed, nothing of the
                        forward pass but rho is kept).
HartreeEnergyAtoms(pos, q)
                        E_H of Gaussian charges.  dE_H/dR_i = -F_i and dE_H/dq_i = phi_i
                        come from the force gather; the backward pass re-solves for V_H
                        inside the library (hartree_forces with no potential), so no grid
                        and no spectrum is stored between forward and backward unless
                        store_potential=True.

Both are first-order only (the backward is not itself differentiable).
"""
from __future__ import annotations

import torch

from .hartree import HartreePlan


def _dV(plan: HartreePlan) -> float:
    n = plan.n
    return plan.cell[0] * plan.cell[1] * plan.cell[2] / (n[0] * n[1] * n[2])


class HartreeEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, plan: HartreePlan):
        rho_c = rho.detach().contiguous()
        _, eh = plan.solve_density(rho_c)
        ctx.plan = plan
        ctx.save_for_backward(rho_c)
        return eh.clone()

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, grad_out):
        (rho,) = ctx.saved_tensors
        plan = ctx.plan
        vh, _ = plan.solve_density(rho)  # recompute V_H; the spectrum is never stored
        grad = vh * (grad_out.to(vh.dtype) * _dV(plan))
        return grad, None


class HartreeEnergyAtoms(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, q, plan: HartreePlan, store_potential: bool = False):
        pos_c = pos.detach().contiguous()
        q_c = q.detach().contiguous()
        vh, eh = plan.solve(pos_c, q_c)
        ctx.plan = plan
        ctx.vh = vh if store_potential else None
        if not store_potential:
            del vh
        ctx.save_for_backward(pos_c, q_c)
        return eh.clone()

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, grad_out):
        pos, q = ctx.saved_tensors
        plan = ctx.plan
        f, phi = plan.forces(pos, q, vh=ctx.vh)  # vh None: the library re-solves internally
        g = grad_out.to(torch.float64)
        return (-f * g if ctx.needs_input_grad[0] else None, phi * g if ctx.needs_input_grad[1] else None, None, None)


def hartree_energy(rho, plan: HartreePlan):
    """E_H of a grid density, differentiable w.r.t. rho."""
    return HartreeEnergy.apply(rho, plan)


def hartree_energy_atoms(pos, q, plan: HartreePlan, store_potential: bool = False):
    """E_H of Gaussian charges, differentiable w.r.t. positions and charges."""
    return HartreeEnergyAtoms.apply(pos, q, plan, store_potential)
