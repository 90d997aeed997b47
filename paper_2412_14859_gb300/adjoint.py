"""The volume history of a run as a differentiable function of the flux field.

``volume_history(sim, phi, nsteps)`` runs ``nsteps`` fused steps from the handle's current state
with the flux field ``phi`` (Eq. relation: each site moves phi(x)/S-bar from red to blue, Eq.
exchange) and returns V(0..nsteps), V the liquid volume sum_x (1 + rho^N)/2.  Its backward pass is
the library's hand-written reverse sweep (``cgevap_adjoint_backward``): segments of
``ckpt_every`` steps are recomputed from checkpoints and the adjoint steps run in reverse, with
the site set of every step held at that of the forward run.  Argument marshalling only: the
steps and the sweep run in the library's kernels.

Typical use, fitting the coefficients a_k of phi = phi0 (1 + sum_k a_k (r/R)^k) to a target
volume-loss history:

    phi = phi0 * (1 + torch.tensordot(a, basis, 1))
    V = volume_history(sim, phi, T)              # sim freshly initialised
    loss = ((V[0] - V[1:] - dV_target) ** 2).sum()
    loss.backward()                              # a.grad
"""
from __future__ import annotations

import torch

from .binding import Sim

__all__ = ["VolumeHistory", "volume_history"]


class VolumeHistory(torch.autograd.Function):
    """V(0..T) of T steps of ``sim`` from its current state, differentiable in the flux field."""

    @staticmethod
    def forward(ctx, phi: torch.Tensor, sim: Sim, nsteps: int, ckpt_every: int):
        if tuple(phi.shape) != tuple(sim.shape):
            raise ValueError(f"phi must have the lattice shape {sim.shape}, got {tuple(phi.shape)}")
        sim.set_flux(0.0, phi.detach().contiguous())
        V = sim.adjoint_forward(int(nsteps), int(ckpt_every))
        ctx.sim = sim
        ctx.phi_dtype = phi.dtype
        return V

    @staticmethod
    def backward(ctx, gV: torch.Tensor):
        dphi = ctx.sim.adjoint_backward(gV.detach().to(torch.float64).contiguous())
        return dphi.to(ctx.phi_dtype), None, None, None


def volume_history(sim: Sim, phi: torch.Tensor, nsteps: int, ckpt_every: int = 64) -> torch.Tensor:
    return VolumeHistory.apply(phi, sim, nsteps, ckpt_every)
