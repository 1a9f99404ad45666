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

Memory.  A segment's step-start states are either kept on the device while
its adjoint steps run (`keep_states`, one state per step of the segment) or,
where they do not fit, each one is recomputed from the segment's checkpoint
just before its adjoint step (quadratic in the segment length, one state of
memory).  Checkpoints are kept on the device or, where they do not fit, in
pinned host memory.  The cotangent of the final state is formed at the end of
the forward pass, so the final state itself is not kept.
"""
from __future__ import annotations

from typing import List, Optional, Tuple

import torch

from .vlasov import VlasovPoisson


def _free_bytes(dev: torch.device) -> int:
    if dev.type != "cuda":
        return 1 << 62          # host tensors: no device-memory limit applies
    free, _total = torch.cuda.mem_get_info(dev)
    return free


def _release_pinned() -> None:
    """Returns the page-locked host memory torch keeps cached after pinned
    tensors are freed (checkpoints of a 49 GB state fill half the host's
    memory) to the system."""
    fn = getattr(torch._C, "_host_emptyCache", None)
    if fn is not None:
        fn()


def _store(t: torch.Tensor, on_device: bool) -> torch.Tensor:
    if on_device:
        return t.clone()
    h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
    h.copy_(t)
    return h


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f0: torch.Tensor, sim: VlasovPoisson, nsteps: int, every: int, kind: int,
                target: Optional[torch.Tensor], keep_states: Optional[bool]):
        f = sim.f
        fbytes = f.numel() * f.element_size()
        nck = (nsteps + every - 1) // every
        # checkpoints on the device if they leave room for the backward's
        # cotangent, the adjoint's three scratch states and one segment state
        ck_dev = _free_bytes(f.device) > (nck + 5) * fbytes
        with torch.no_grad():
            f.copy_(f0)
            sim.refresh_field()
            ckpts: List[Tuple[torch.Tensor, torch.Tensor]] = []
            # one call per segment: between two checkpoints the steps run as
            # the fused body (K2^n and K1^{n+1} in one pass over f)
            for n0 in range(0, nsteps, every):
                ckpts.append((_store(f, ck_dev), sim.field()[2]))
                sim.step(min(every, nsteps - n0))
            lam_f = torch.empty_like(f)
            J = sim.functional(kind, lam_f, target)
        ctx.sim, ctx.nsteps, ctx.every = sim, nsteps, every
        ctx.ckpts, ctx.lam_f, ctx.keep = ckpts, lam_f, keep_states
        return f0.new_tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ: torch.Tensor):
        sim: VlasovPoisson = ctx.sim
        f = sim.f
        fbytes = f.numel() * f.element_size()
        if f.is_cuda:
            # the adjoint's scratch states are allocated by the library, outside
            # torch's caching allocator: blocks torch keeps cached would not be
            # available to it
            torch.cuda.empty_cache()
        with torch.no_grad():
            lam_f = ctx.lam_f
            lam_g = torch.zeros((3,) + tuple(sim.cfg.n), dtype=torch.float64, device=f.device)
            nsteps, every = ctx.nsteps, ctx.every
            for s in reversed(range(len(ctx.ckpts))):
                n0 = s * every
                n1 = min(n0 + every, nsteps)
                fc, gc = ctx.ckpts[s]
                keep = ctx.keep
                if keep is None:
                    keep = _free_bytes(f.device) > (n1 - n0 + 3) * fbytes
                if keep:
                    # states of the segment: f^n, g^n for n0 <= n < n1
                    f.copy_(fc)
                    sim.set_accel(gc)
                    # every step-start state is kept, so the steps run one
                    # call each (inside a fused body the state between two
                    # steps is never in memory)
                    states = []
                    for n in range(n0, n1):
                        states.append((f.clone(), sim.field()[2]))
                        if n + 1 < n1:          # f^{n1} is not needed
                            sim.step(1)
                    for fs, gs in reversed(states):
                        sim.adjoint_step(fs, gs, lam_f, lam_g)
                    del states
                else:
                    # f^n recomputed from the checkpoint before each adjoint step;
                    # the context's own f serves as the step-start state
                    for n in reversed(range(n0, n1)):
                        f.copy_(fc)
                        sim.set_accel(gc)
                        if n > n0:
                            sim.step(n - n0)
                        sim.adjoint_step(f, sim.field()[2], lam_f, lam_g)
            # g^0 = -grad phi[rho(f^0)]
            sim.field_adjoint(lam_g, lam_f)
            on_host = any(not fc.is_cuda for fc, _ in ctx.ckpts)
            ctx.ckpts = None
            if on_host:
                _release_pinned()
            # the cotangent itself becomes the gradient (no second array of
            # f's size: at 48^6 that would not fit beside the adjoint's scratch)
            lam_f.mul_(gJ.to(lam_f.dtype))
        ctx.lam_f = None
        return lam_f, None, None, None, None, None, None


def trajectory_functional(f0: torch.Tensor, sim: VlasovPoisson, nsteps: int, every: int = 10,
                          kind: int = 0, target: Optional[torch.Tensor] = None,
                          keep_states: Optional[bool] = None) -> torch.Tensor:
    """J(f(t_n)) after nsteps split steps from f0 (kind 0: field energy U,
    kind 1: density misfit 1/2 sum (rho - target)^2 dV), differentiable in f0.
    keep_states: keep each segment's states on the device (True), recompute
    them from the checkpoint (False), or decide from the free memory (None)."""
    return _Trajectory.apply(f0, sim, int(nsteps), int(every), int(kind), target, keep_states)
