"""torch.autograd.Function over the density + smoothing-length solve +
force pipeline, with the hand-written adjoint kernels as its backward.

Forward:  pos (N,3) float64, m (N,), u (N,), vel (N,3) or None
          -> rho (N,), acc (N,3), dudt (N,)  [float32, caller order]
Backward: dL/drho, dL/dacc, dL/ddudt -> dL/dpos (float64), dL/dm, dL/du
The smoothing lengths are an internal, implicitly differentiated quantity
(h solves N_i(h_i, x) = N_ngb), so they do not appear as an input.
"""
from __future__ import annotations

import torch

from .sph import SPH


class SPHDensityForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, m, u, vel, sph: SPH, box: float, h_guess):
        sph.build(pos, box=box, h_guess=h_guess)
        d = sph.density(m)
        acc, dudt, _ = sph.force(u, vel)
        ctx.sph = sph
        ctx.pos_dtype = pos.dtype
        ctx.mark_non_differentiable(d["h"])
        return d["rho"], acc, dudt, d["h"]

    @staticmethod
    def backward(ctx, g_rho, g_acc, g_dudt, g_h):
        sph = ctx.sph
        g_pos, g_m, g_u = sph.adjoint(g_rho, g_acc, g_dudt)
        return g_pos.to(ctx.pos_dtype), g_m, g_u, None, None, None, None


def sph_density_force(pos, m, u, vel=None, sph: SPH | None = None, box: float = 1.0,
                      h_guess=None):
    """Differentiable SPH step: returns (rho, acc, dudt, h)."""
    sph = sph or SPH()
    return SPHDensityForce.apply(pos, m, u, vel, sph, box, h_guess)
