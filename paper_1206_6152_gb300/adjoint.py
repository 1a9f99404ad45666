"""Gradients of a final-time functional through the split step.

The discrete adjoint (include/vp.h: vp_adjoint_step, vp_field_adjoint,
vp_functional) sits behind a torch.autograd.Function.  The forward runs n
steps from f0 and keeps a checkpoint (f, g) every `every` steps; the backward
walks the segments in reverse, recomputes the states of a segment from its
checkpoint, and applies the adjoint step by step.  The initial acceleration is
g0 = field(f0), so its cotangent is finally sent back into f0 as well.

    J = trajectory_functional(f0, sim, nsteps, every, kind, target)
    J.backward()          # f0.grad = dJ/df0

f0 may itself be a function of parameters (e.g. mode amplitudes); torch's own
autograd carries the chain rule from dJ/df0 to them.
"""
from __future__ import annotations

from typing import List, Optional, Tuple

import torch

from .vlasov import VlasovPoisson


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f0: torch.Tensor, sim: VlasovPoisson, nsteps: int, every: int, kind: int,
                target: Optional[torch.Tensor]):
        f = sim.f
        with torch.no_grad():
            f.copy_(f0)
            sim.refresh_field()
            ckpts: List[Tuple[torch.Tensor, torch.Tensor]] = []
            for n in range(nsteps):
                if n % every == 0:
                    ckpts.append((f.clone(), sim.field()[2]))
                sim.step(1)
            lam_dummy = torch.empty_like(f)
            J = sim.functional(kind, lam_dummy, target)
        ctx.sim, ctx.nsteps, ctx.every, ctx.kind, ctx.target = sim, nsteps, every, kind, target
        ctx.ckpts = ckpts
        ctx.final = f.clone()
        return f0.new_tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ: torch.Tensor):
        sim: VlasovPoisson = ctx.sim
        f = sim.f
        with torch.no_grad():
            f.copy_(ctx.final)
            lam_f = torch.empty_like(f)
            sim.functional(ctx.kind, lam_f, ctx.target)
            lam_g = torch.zeros((3,) + tuple(sim.cfg.n), dtype=torch.float64, device=f.device)
            nsteps, every = ctx.nsteps, ctx.every
            for s in reversed(range(len(ctx.ckpts))):
                n0 = s * every
                n1 = min(n0 + every, nsteps)
                fc, gc = ctx.ckpts[s]
                # states of the segment: f^n, g^n for n0 <= n < n1
                f.copy_(fc)
                sim.set_accel(gc)
                states = []
                for _ in range(n0, n1):
                    states.append((f.clone(), sim.field()[2]))
                    sim.step(1)
                for fs, gs in reversed(states):
                    sim.adjoint_step(fs, gs, lam_f, lam_g)
                del states
            # g^0 = -grad phi[rho(f^0)]
            sim.field_adjoint(lam_g, lam_f)
        grad = lam_f * gJ.to(lam_f.dtype)
        return grad, None, None, None, None, None


def trajectory_functional(f0: torch.Tensor, sim: VlasovPoisson, nsteps: int, every: int = 10,
                          kind: int = 0, target: Optional[torch.Tensor] = None) -> torch.Tensor:
    """J(f(t_n)) after nsteps split steps from f0 (kind 0: field energy U,
    kind 1: density misfit 1/2 sum (rho - target)^2 dV), differentiable in f0."""
    return _Trajectory.apply(f0, sim, int(nsteps), int(every), int(kind), target)
