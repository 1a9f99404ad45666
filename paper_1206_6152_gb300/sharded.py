"""Position space cut into slabs along x, one slab per GPU.

The decomposition of Sec. 2.3: position space is divided among the
processes and velocity space is kept whole, so the kicks and the y and z
drifts of a slab need nothing from other slabs.  The x drift does: a cell's
update reads cells up to floor(|alpha|) + 2 upwind and one downwind, so each
slab receives that many ghost planes from each neighbour (the periodic wrap
included), and the slope corrector's f_inf is the maximum of the whole x line,
so the per-slab maxima are reduced over the slabs (Sec. 4 discusses the cost
of that global maximum).  The field is solved on the whole grid on every GPU
from the gathered density (the FFT is not distributed, as in Sec. 2.3), and
each slab keeps its part of g.

Per step (Eq. integration, as the single-GPU step):

    dt from g^n (the previous field solve)
    K1: vx, vy, vz sweeps (dt/2), slab-local
    z, y drifts (dt), slab-local
    line maxima along x -> all-reduce max;  G edge planes -> neighbours
    x drift (dt) of each slab with its ghost planes and the whole lines' maxima
    density of each slab -> all-gather -> phi, g^{n+1} and the next dt
    K2: vx, vy, vz sweeps (dt/2) with g^{n+1}  (with the next step's K1 in
        the same passes, as in the single-GPU step)

Each slab's work goes through a backend (`LibrarySlab`: the CUDA library's
slab context and a field-only context of the whole grid); the exchanges go
through an `Exchange`: `DistExchange` over a torch.distributed group (one slab
per rank: all_reduce, all_gather, point-to-point halo planes; NCCL for CUDA
tensors, gloo for host tensors) or `LocalExchange` for several slabs held by
one process (direct copies).  Periodic position space; the x planes must
divide evenly among the slabs.
"""
from __future__ import annotations

import ctypes
import math
from typing import List, Optional, Sequence, Tuple

import torch

from . import _lib
from ._lib import check, vp_config
from .vlasov import VlasovPoisson

Tensor = torch.Tensor


# ---------------------------------------------------------------------------
# exchanges
# ---------------------------------------------------------------------------

class LocalExchange:
    """All slabs in this process, in x order (slab r holds planes
    [r Nx/R, (r+1) Nx/R)); the collectives are direct copies."""

    def allreduce_max(self, parts: Sequence[Tensor]) -> List[Tensor]:
        m = parts[0].clone()
        for p in parts[1:]:
            torch.maximum(m, p.to(m.device), out=m)
        return [m.to(p.device) for p in parts]

    def allgather_x(self, parts: Sequence[Tensor]) -> List[Tensor]:
        whole = torch.cat([p.to(parts[0].device) for p in parts], dim=0)
        return [whole.to(p.device) for p in parts]

    def halos(self, edges: Sequence[Tuple[Tensor, Tensor]]) -> List[Tuple[Tensor, Tensor]]:
        """edges[r] = (first G planes, last G planes) of slab r; returns per
        slab (planes below it, planes above it) of the periodic box."""
        R = len(edges)
        return [(edges[(r - 1) % R][1].to(edges[r][0].device).contiguous(),
                 edges[(r + 1) % R][0].to(edges[r][0].device).contiguous()) for r in range(R)]


class DistExchange:
    """One slab per rank of a torch.distributed group; slab r holds planes
    [r Nx/W, (r+1) Nx/W)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def _peer(self, r: int) -> int:
        return self.dist.get_global_rank(self.group, r) if self.group is not None else r

    def allreduce_max(self, parts: Sequence[Tensor]) -> List[Tensor]:
        (p,) = parts
        m = p.clone()
        self.dist.all_reduce(m, op=self.dist.ReduceOp.MAX, group=self.group)
        return [m]

    def allgather_x(self, parts: Sequence[Tensor]) -> List[Tensor]:
        (p,) = parts
        p = p.contiguous()
        out = [torch.empty_like(p) for _ in range(self.world)]
        self.dist.all_gather(out, p, group=self.group)
        return [torch.cat(out, dim=0)]

    def halos(self, edges: Sequence[Tuple[Tensor, Tensor]]) -> List[Tuple[Tensor, Tensor]]:
        ((first, last),) = edges
        if self.world == 1:
            return [(last.clone(), first.clone())]
        dist = self.dist
        prev = self._peer((self.rank - 1) % self.world)
        nxt = self._peer((self.rank + 1) % self.world)
        lo = torch.empty_like(last)
        hi = torch.empty_like(first)
        # my first planes are the lower neighbour's upper ghosts (tag 1), my
        # last planes the upper neighbour's lower ghosts (tag 2); with two
        # ranks both go to the same peer, told apart by tag (gloo) or by the
        # order of the operations (NCCL)
        ops = [dist.P2POp(dist.isend, first.contiguous(), prev, self.group, 1),
               dist.P2POp(dist.isend, last.contiguous(), nxt, self.group, 2),
               dist.P2POp(dist.irecv, hi, nxt, self.group, 1),
               dist.P2POp(dist.irecv, lo, prev, self.group, 2)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        return [(lo, hi)]


# ---------------------------------------------------------------------------
# the library's slab
# ---------------------------------------------------------------------------

def slab_config(cfg: vp_config, x0: int, nx: int) -> vp_config:
    """The configuration of the slab of planes [x0, x0 + nx) of cfg's box
    (same cell widths)."""
    c = vp_config()
    ctypes.memmove(ctypes.byref(c), ctypes.byref(cfg), ctypes.sizeof(vp_config))
    dx = (cfg.box_hi[0] - cfg.box_lo[0]) / cfg.n[0]
    c.n[0] = nx
    c.box_lo[0] = cfg.box_lo[0] + x0 * dx
    c.box_hi[0] = cfg.box_lo[0] + (x0 + nx) * dx
    return c


class LibrarySlab:
    """One slab on one GPU: the library's context of the slab (kicks, y and z
    drifts, the ghosted x drift, line maxima, density) and a field-only
    context of the whole grid (the replicated field solve and dt)."""

    def __init__(self, cfg: vp_config, x0: int, f_slab: Tensor,
                 stream: Optional[torch.cuda.Stream] = None):
        if cfg.space_bc != 0:
            raise ValueError("slabs need periodic position space")
        self.lib = _lib.load()
        self.cfg = cfg
        self.x0 = x0
        self.nx = int(f_slab.shape[0])
        self.sim = VlasovPoisson(slab_config(cfg, x0, self.nx), f_slab, stream)
        self.f = f_slab
        self.n = tuple(cfg.n)
        self._fctx = ctypes.c_void_p()
        with torch.cuda.device(f_slab.device):
            check(self.lib.vp_field_init(ctypes.byref(cfg), ctypes.c_void_p(self.sim.stream.cuda_stream),
                                         ctypes.byref(self._fctx)), "vp_field_init")

    def close(self):
        if self._fctx:
            self.lib.vp_destroy(self._fctx)
            self._fctx = ctypes.c_void_p()
        self.sim.close()

    def kick(self, tau: float, tau_next: float = 0.0) -> None:
        """A half kick of duration tau; with tau_next, the next step's first
        half kick after it (same g), in the fused passes of the step."""
        check(self.lib.vp_kick(self.sim._ctx, float(tau), float(tau_next)), "vp_kick")

    def drift_yz(self, tau: float) -> None:
        check(self.lib.vp_drift_yz(self.sim._ctx, float(tau)), "vp_drift_yz")

    def line_max_x(self) -> Tensor:
        out = torch.empty(self.f.shape[1:], dtype=self.f.dtype, device=self.f.device)
        check(self.lib.vp_line_max_x(self.sim._ctx, ctypes.c_void_p(out.data_ptr())), "vp_line_max_x")
        return out

    def planes(self, lo: int, hi: int) -> Tensor:
        return self.f[lo:hi].clone()

    def drift_x(self, tau: float, glo: Tensor, ghi: Tensor, nghost: int, lmax: Tensor) -> None:
        for t, name in ((glo, "ghost_lo"), (ghi, "ghost_hi")):
            if (t.device != self.f.device or t.dtype != self.f.dtype or not t.is_contiguous()
                    or tuple(t.shape) != (nghost,) + tuple(self.f.shape[1:])):
                raise ValueError(f"{name} must be {nghost} contiguous planes of f on its device")
        if (lmax.device != self.f.device or lmax.dtype != self.f.dtype or not lmax.is_contiguous()
                or tuple(lmax.shape) != tuple(self.f.shape[1:])):
            raise ValueError("lmax must be one contiguous plane of f on its device")
        check(self.lib.vp_drift_x_ghosted(self.sim._ctx, float(tau), ctypes.c_void_p(glo.data_ptr()),
                                          ctypes.c_void_p(ghi.data_ptr()), int(nghost),
                                          ctypes.c_void_p(lmax.data_ptr())), "vp_drift_x_ghosted")

    def density(self) -> Tensor:
        return self.sim.density()

    def field(self, rho: Tensor) -> Tuple[Tensor, float]:
        rho = rho.to(device=self.f.device, dtype=torch.float64).contiguous()
        if tuple(rho.shape) != self.n:
            raise ValueError(f"rho must have shape {self.n}")
        g = torch.empty((3,) + self.n, dtype=torch.float64, device=self.f.device)
        dt = ctypes.c_double()
        check(self.lib.vp_field_solve(self._fctx, ctypes.c_void_p(rho.data_ptr()),
                                      ctypes.c_void_p(g.data_ptr()), ctypes.byref(dt)),
              "vp_field_solve")
        return g, dt.value

    def set_accel(self, g_slab: Tensor) -> None:
        self.sim.set_accel(g_slab.contiguous())

    def vmax_x(self) -> float:
        """max |v_x| over the velocity cell centres."""
        dv = (self.cfg.vhi[0] - self.cfg.vlo[0]) / self.cfg.nv[0]
        return max(abs(self.cfg.vlo[0] + 0.5 * dv), abs(self.cfg.vhi[0] - 0.5 * dv))

    def dx(self) -> float:
        return (self.cfg.box_hi[0] - self.cfg.box_lo[0]) / self.cfg.n[0]


# ---------------------------------------------------------------------------
# the step
# ---------------------------------------------------------------------------

class ShardedStep:
    """The split step over x slabs.  `slabs` are this process's slabs in x
    order (all of them with a LocalExchange, its own one with a
    DistExchange); each provides kick(tau[, tau_next]), drift_yz,
    line_max_x, planes, drift_x, density, field, set_accel, vmax_x, dx and
    the attributes x0, nx.  Within one call of step(n) the second half kick
    of a step and the first of the next run together (they share g^{n+1}),
    as in the single-context step."""

    def __init__(self, slabs: Sequence, exchange):
        self.slabs = list(slabs)
        self.ex = exchange
        self.t = 0.0
        self.dt = self._field()

    def _field(self) -> float:
        """Gathers the density, solves for the field on every slab's side and
        hands each slab its part of g; returns the dt of that g."""
        rhos = self.ex.allgather_x([s.density() for s in self.slabs])
        dt = None
        for s, rho in zip(self.slabs, rhos):
            g, dt = s.field(rho)
            s.set_accel(g[:, s.x0:s.x0 + s.nx])
        return dt

    def nghost(self, dt: float) -> int:
        s = self.slabs[0]
        G = int(math.floor(s.vmax_x() * dt / s.dx())) + 2
        if any(G > b.nx for b in self.slabs):
            raise ValueError(f"an x shift of {G - 2} cells needs slabs of at least {G} planes")
        return G

    def step(self, nsteps: int = 1) -> float:
        for n in range(nsteps):
            dt = self.dt
            if n == 0:
                for s in self.slabs:
                    s.kick(0.5 * dt)                     # K1 of the first step
            for s in self.slabs:
                s.drift_yz(dt)
            lmax = self.ex.allreduce_max([s.line_max_x() for s in self.slabs])
            G = self.nghost(dt)
            halos = self.ex.halos([(s.planes(0, G), s.planes(s.nx - G, s.nx)) for s in self.slabs])
            for s, (lo, hi), m in zip(self.slabs, halos, lmax):
                s.drift_x(dt, lo, hi, G, m)
            self.dt = self._field()
            for s in self.slabs:
                if n + 1 < nsteps:
                    s.kick(0.5 * dt, 0.5 * self.dt)      # K2 of this step, K1 of the next
                else:
                    s.kick(0.5 * dt)                     # K2 of the last step
            self.t += dt
        return self.t
