"""torch.autograd.Function wrappers of the tree forces and of a leap-frog run.

Both hold the tree and interaction lists of their forward pass fixed in the
backward pass (the derivative of the forward map for those lists), and both
run entirely in the CUDA library: the forward through tree_build /
tree_forces / tree_run, the backward through tree_forces_vjp / tree_run_vjp.
The TreeGravity object passed in must not be rebuilt between a forward
and its backward.
"""
from __future__ import annotations

import torch

from .gravity import TreeGravity


class TreeForces(torch.autograd.Function):
    """acc (3, N) float32, pot (N,) float32 = TreeForces.apply(pos, mass, grav, theta, eps)
    with pos (3, N) and mass (N,) float64 CUDA tensors."""

    @staticmethod
    def forward(ctx, pos, mass, grav: TreeGravity, theta: float, eps: float):
        grav.build(pos.detach().contiguous(), mass.detach().contiguous())
        acc, pot = grav.forces(theta, eps)
        ctx.grav = grav
        return acc, pot

    @staticmethod
    def backward(ctx, gacc, gpot):
        gacc = torch.zeros((3, ctx.grav.n), dtype=torch.float32, device=gpot.device) if gacc is None \
            else gacc.to(torch.float32)
        gpot = None if gpot is None else gpot.to(torch.float32)
        gpos, gmass = ctx.grav.forces_vjp(gacc, gpot)
        return gpos, gmass, None, None, None


class LeapfrogRun(torch.autograd.Function):
    """pos_K, vel_K = LeapfrogRun.apply(pos0, vel0, mass, grav, nsteps, dt, ckpt_every):
    nsteps kick-drift-kick steps (FP64 state) with checkpoints every
    ckpt_every steps; the backward re-integrates each segment and applies
    the force VJP at every position."""

    @staticmethod
    def forward(ctx, pos0, vel0, mass, grav: TreeGravity, nsteps: int, dt: float, ckpt_every: int):
        grav.build(pos0.detach().contiguous(), mass.detach().contiguous())
        grav.set_velocities(vel0.detach().contiguous())
        grav.run(nsteps, dt, ckpt_every)
        pos, vel, _ = grav.state()
        ctx.grav = grav
        return pos, vel

    @staticmethod
    def backward(ctx, xbar, vbar):
        n = ctx.grav.n
        dev = xbar.device if xbar is not None else vbar.device
        xbar = torch.zeros((3, n), dtype=torch.float64, device=dev) if xbar is None else xbar.to(torch.float64)
        vbar = torch.zeros((3, n), dtype=torch.float64, device=dev) if vbar is None else vbar.to(torch.float64)
        x0, v0, m0 = ctx.grav.run_vjp(xbar, vbar)
        return x0, v0, m0, None, None, None, None
