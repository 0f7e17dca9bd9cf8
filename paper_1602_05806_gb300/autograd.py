"""torch.autograd interface of the time step with the library's hand-written
adjoint (sdg_step_adjoint).

    U_T, P_T = steps(h, U0, P0, nu, nsteps)

runs nsteps steps of the handle from (U0, P0) and returns the final state;
backward() runs the adjoint steps in reverse from the velocity checkpointed
at the start of every step (the stages are recomputed inside the library),
giving gradients with respect to U0, P0 and the viscosity nu (a 0-d tensor
whose value must equal the handle's nu).  All arithmetic runs in libsdg.
"""
from __future__ import annotations

import torch

from . import sdg

__all__ = ["steps"]


class _Steps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, nsteps, nu, P0, *U0):
        if int(nsteps) < 1:
            raise ValueError("nsteps must be >= 1")
        if abs(float(nu) - float(h.nu)) > 1e-15 * max(1.0, abs(float(h.nu))):
            raise ValueError("nu must equal the viscosity the handle was created with")
        U0 = [u.detach().contiguous() for u in U0]
        h.set_state(U0, P0.detach().contiguous())
        ckpt = []
        for _ in range(int(nsteps)):
            Uk = [torch.empty_like(U0[0]) for _ in range(h.dim)]
            Pk = torch.empty_like(U0[0])
            h.get_state(Uk, Pk)
            ckpt.append(Uk)
            info = h.step(1)
            if info["status"] != sdg.SDG_OK:
                raise sdg.SDGError(info["status"], "step failed in the forward pass")
        UT = [torch.empty_like(U0[0]) for _ in range(h.dim)]
        PT = torch.empty_like(U0[0])
        h.get_state(UT, PT)
        ctx.h, ctx.ckpt = h, ckpt
        ctx.nu_meta = (nu.dtype, nu.device)
        return (PT, *UT)

    @staticmethod
    def backward(ctx, gP, *gU):
        h = ctx.h
        like = ctx.ckpt[0][0] if ctx.ckpt else None
        lamU = [(g.detach().clone().contiguous() if g is not None else torch.zeros_like(like)) for g in gU]
        lamP = gP.detach().clone().contiguous() if gP is not None else torch.zeros_like(lamU[0])
        dnu = 0.0
        for Uk in reversed(ctx.ckpt):
            dnu += h.step_adjoint(Uk, lamU, lamP)
        dtype, device = ctx.nu_meta
        return (None, None, torch.tensor(dnu, dtype=dtype, device=device), lamP, *lamU)


def steps(h, U0, P0, nu, nsteps):
    """(U_T list, P_T) after nsteps steps of handle h from (U0, P0);
    differentiable in U0, P0 and nu (see the module docstring)."""
    out = _Steps.apply(h, int(nsteps), nu, P0, *U0)
    return list(out[1:]), out[0]
