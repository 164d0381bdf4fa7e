"""torch.autograd.Function over the density + smoothing-length solve +
force pipeline, with the hand-written adjoint kernels as its backward.

Forward:  pos (N,3) float64, m (N,), u (N,), vel (N,3) or None
          -> rho (N,), acc (N,3), dudt (N,)  [float32, caller order]
Backward: dL/drho, dL/dacc, dL/ddudt -> dL/dpos (float64), dL/dm, dL/du
The smoothing lengths are an internal, implicitly differentiated quantity
(h solves N_i(h_i, x) = N_ngb), so they do not appear as an input.
Velocities are treated as constants: the adjoint kernels give no
gradient for them, so a vel that requires grad is refused.

The adjoint reads the forward state kept in the SPH context.  A context
serves one differentiable forward at a time: backward raises if another
build / density / force call has replaced that state since (the context's
state generation changed).
"""
from __future__ import annotations

import torch

from .sph import SPH


class SPHDensityForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, m, u, vel, sph: SPH, box: float, h_guess):
        if vel is not None and vel.requires_grad:
            raise ValueError("sph_density_force: velocities are constants of the adjoint; "
                             "pass vel.detach()")
        sph.build(pos, box=box, h_guess=h_guess)
        d = sph.density(m)
        acc, dudt, _ = sph.force(u, vel)
        ctx.sph = sph
        ctx.gen = sph.generation()
        ctx.pos_dtype = pos.dtype
        ctx.mark_non_differentiable(d["h"])
        return d["rho"], acc, dudt, d["h"]

    @staticmethod
    def backward(ctx, g_rho, g_acc, g_dudt, g_h):
        sph = ctx.sph
        if sph.generation() != ctx.gen:
            raise RuntimeError("sph_density_force: the SPH context ran another forward after this "
                               "one; its adjoint state is gone (use one context per pending "
                               "backward)")
        g_pos, g_m, g_u = sph.adjoint(g_rho, g_acc, g_dudt)
        return g_pos.to(ctx.pos_dtype), g_m, g_u, None, None, None, None


def sph_density_force(pos, m, u, vel=None, sph: SPH | None = None, box: float = 1.0,
                      h_guess=None):
    """Differentiable SPH step: returns (rho, acc, dudt, h)."""
    sph = sph or SPH()
    return SPHDensityForce.apply(pos, m, u, vel, sph, box, h_guess)
