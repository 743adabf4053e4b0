"""torch.autograd.Function around dem_adjoint.

J(theta) is the mean over all parcels of the reduction degree gained over n sub-steps of the
frozen-position drag-heat-reaction map, theta = (k0[3], Ea[3]) of the three reactions
(eq (2-13); the parameters whose effect Sec. 5 studies). Forward sets the kinetics on the
context and runs the library's adjoint (forward sweep with checkpoints, recomputation,
hand-written reverse sweep); backward returns the stored gradient times the incoming one.
"""
from __future__ import annotations

import numpy as np
import torch


class ReductionDegree(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, dem_context, nsteps: int, ckpt_every: int):
        p = params.detach().to("cpu", torch.float64).numpy()
        dem_context.dem_set_kinetics(p[:3], p[3:])
        J, g = dem_context.dem_adjoint(int(nsteps), int(ckpt_every))
        ctx.save_for_backward(torch.from_numpy(np.asarray(g, dtype=np.float64)).to(params.device))
        return torch.tensor(J, dtype=torch.float64, device=params.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g.to(grad_out.dtype), None, None, None


def reduction_degree(params: torch.Tensor, dem_context, nsteps: int = 2000, ckpt_every: int = 100):
    """Differentiable J(k0, Ea); params is a 6-vector (k0[3], Ea[3])."""
    return ReductionDegree.apply(params, dem_context, nsteps, ckpt_every)


class ReductionDegreeCurves(torch.autograd.Function):
    """The bed reduction-degree curves J_obs (n_obs, n_beds) of the frozen-position map
    observed after obs_steps sub-steps, as a function of theta = (k0[3], Ea[3]); backward
    runs the library's reverse sweep once with the incoming gradient as the observation
    weights (dem_adjoint_obs)."""

    @staticmethod
    def forward(ctx, params, dem_context, nsteps: int, obs_steps, ckpt_every: int):
        p = params.detach().to("cpu", torch.float64).numpy()
        dem_context.dem_set_kinetics(p[:3], p[3:])
        Jo, _ = dem_context.dem_adjoint_obs(int(nsteps), obs_steps, None, int(ckpt_every))
        ctx.dem = (dem_context, int(nsteps), list(obs_steps), int(ckpt_every), p)
        return torch.from_numpy(Jo).to(params.device)

    @staticmethod
    def backward(ctx, grad_out):
        dem, nsteps, obs, ck, p = ctx.dem
        dem.dem_set_kinetics(p[:3], p[3:])
        w = grad_out.detach().to("cpu", torch.float64).numpy()
        _, g = dem.dem_adjoint_obs(nsteps, obs, w, ck)
        return torch.from_numpy(g).to(grad_out.device, grad_out.dtype), None, None, None, None


def reduction_degree_curves(params: torch.Tensor, dem_context, nsteps: int, obs_steps, ckpt_every: int = 200):
    """Differentiable bed reduction-degree curves J_obs(k0, Ea), (n_obs, n_beds)."""
    return ReductionDegreeCurves.apply(params, dem_context, nsteps, obs_steps, ckpt_every)
