"""The pseudofermion action as a differentiable torch function.

S(U) = sum_i r_i Re(b^dag x_i),  x_i = (m^2 + sigma_i - D_eo D_oe)^-1 b  (Eq. shift_eo).
forward runs the multi-shift CG and the action's reduction (libstg); backward runs the hand-written
adjoint kernel (stg_fermion_force, kind 1), which returns W^dag per link:
the gradient in torch's convention for a real loss of complex inputs,
dS/dRe U + i dS/dIm U, since dS = Re tr(dU W).
"""
from __future__ import annotations

import torch

from .api import Gauge, Lattice, fermion_force, mscg, pseudofermion_action_value as _action, stout_force, stout_smear


class PseudofermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, links, b, lattice: Lattice, shifts, residues, mass: float, tol: float = 1e-12):
        g = Gauge(lattice, links.detach(), "f64", 18)
        x, _ = mscg(g, b.detach(), shifts, mass, tol=tol)
        s = _action(lattice, b.detach(), x, residues)
        ctx.save_for_backward(x)
        ctx.gauge = g
        ctx.residues = list(residues)
        ctx.shape = links.shape
        return torch.as_tensor(s, dtype=torch.float64, device=links.device)

    @staticmethod
    def backward(ctx, grad_s):
        (x,) = ctx.saved_tensors
        w_dag = fermion_force(ctx.gauge, ctx.residues, x, kind=1)
        return (grad_s * w_dag).reshape(ctx.shape), None, None, None, None, None, None


def pseudofermion_action(links, b, lattice, shifts, residues, mass, tol=1e-12):
    """S(U) with autograd support with respect to the links (complex128 [4, V, 3, 3] on cuda)."""
    return PseudofermionAction.apply(links, b, lattice, shifts, residues, mass, tol)


class StoutSmear(torch.autograd.Function):
    """U^(0) -> U^(nstep) by nstep stout steps (stg_stout_smear); backward pulls the incoming
    gradient back through the steps with the hand-written chain-rule kernels (stg_stout_force,
    kind 1), in the same convention."""

    @staticmethod
    def forward(ctx, links, lattice: Lattice, rho: float, nstep: int):
        u = links.detach()
        levels = stout_smear(lattice, u, rho, nstep)
        ctx.save_for_backward(u, levels)
        ctx.lattice = lattice
        ctx.rho = float(rho)
        ctx.shape = links.shape
        return levels[-1].clone().reshape(links.shape)

    @staticmethod
    def backward(ctx, grad_out):
        u, levels = ctx.saved_tensors
        g = stout_force(ctx.lattice, u, levels, ctx.rho, grad_out.contiguous(), kind=1)
        return g.reshape(ctx.shape), None, None, None


def stout_smear_links(links, lattice, rho, nstep):
    """U^(nstep)(U^(0)) with autograd support (complex128 [4, V, 3, 3] on cuda)."""
    return StoutSmear.apply(links, lattice, rho, nstep)
