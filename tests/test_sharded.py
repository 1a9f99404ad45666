"""Position space in x slabs (the decomposition of Sec. 2.3), on the CPU: the
orchestration of paper_1206_6152_gb300/sharded.py -- halo planes of
floor(|alpha|) + 2 cells from each neighbour with the periodic wrap, the
all-reduce of the per-line maxima f_inf, the all-gather of the density for
the replicated field solve, the dt of the gathered field -- run with the FP64
oracle as each slab's arithmetic, against the oracle's single-process step:
bit for bit.  The slabs exchange by direct copies in one process
(LocalExchange) and as gloo ranks (DistExchange, world sizes 2 and 3)."""
import math
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import vp_oracle as O  # noqa: E402
from paper_1206_6152_gb300 import inputs as I  # noqa: E402
from paper_1206_6152_gb300.sharded import DistExchange, LocalExchange, ShardedStep  # noqa: E402


class OracleSlab:
    """The planes [x0, x0 + nx) of a workload's box with the oracle's
    arithmetic behind the slab interface of sharded.py (host tensors)."""

    def __init__(self, w, x0, nx, f0):
        self.w = w
        self.x0, self.nx = x0, nx
        self.grid = O.Grid.of(w)
        dx = self.grid.dx[0]
        self.slab = O.Grid((nx,) + tuple(w.n[1:]), w.nv,
                           (w.box_lo[0] + x0 * dx,) + tuple(w.box_lo[1:]),
                           (w.box_lo[0] + (x0 + nx) * dx,) + tuple(w.box_hi[1:]), w.vlo, w.vhi)
        self.f = np.array(f0[x0:x0 + nx], dtype=np.float64)
        self.g = None

    def kick(self, tau, tau_next=0.0):
        for t in (tau, tau_next) if tau_next else (tau,):
            for a in range(3):
                O.sweep(self.f, 3 + a, self.g[a], t, self.grid.dv[a], False)

    def drift_yz(self, tau):
        for a in (2, 1):
            O.sweep(self.f, a, self.grid.vc(a), tau, self.grid.dx[a], True)

    def line_max_x(self):
        return torch.from_numpy(np.maximum(self.f.max(axis=0), 0.0))

    def planes(self, lo, hi):
        return torch.from_numpy(self.f[lo:hi].copy())

    def drift_x(self, tau, glo, ghi, nghost, lmax):
        assert glo.shape[0] == nghost == ghi.shape[0]
        self.f = O.sweep_x_ghosted(self.f, glo.numpy(), ghi.numpy(), self.grid.vc(0), tau,
                                   self.grid.dx[0], lmax.numpy())

    def density(self):
        return torch.from_numpy(O.density(self.f, self.slab))

    def field(self, rho):
        phi = O.poisson(rho.numpy(), self.grid, self.w.G, "periodic")
        g = O.force(phi, self.grid, "periodic")
        dt = self.w.dt_fixed if self.w.dt_fixed > 0 else O.timestep(g, self.grid, self.w.courant)
        return torch.from_numpy(g), dt

    def set_accel(self, g_slab):
        self.g = np.ascontiguousarray(g_slab.numpy())

    def vmax_x(self):
        return max(abs(self.w.vlo[0] + 0.5 * self.grid.dv[0]), abs(self.w.vhi[0] - 0.5 * self.grid.dv[0]))

    def dx(self):
        return self.grid.dx[0]


def workload(fixed_dt=False):
    w = I.small_maxwell(n=(12, 4, 5), nv=(6, 4, 5), dtype="f64", amp=0.3, G=25.0)
    w = w.replace(box_lo=(-0.5, -0.2, -0.25), box_hi=(0.5, 0.2, 0.25))
    if fixed_dt:
        # x shifts of up to 2.6 cells: four ghost planes
        dx = 1.0 / 12
        vmax = max(abs(w.vlo[0] + 0.5 * (w.vhi[0] - w.vlo[0]) / 6),
                   abs(w.vhi[0] - 0.5 * (w.vhi[0] - w.vlo[0]) / 6))
        w = w.replace(dt_fixed=2.6 * dx / vmax)
    return w


def reference(w, nsteps):
    ref = O.Simulation(I.initial_condition(w, np.float64), O.Grid.of(w), O.Params.of(w))
    ref.step(nsteps)
    return ref


@pytest.mark.parametrize("nslabs", [1, 2, 3])
@pytest.mark.parametrize("fixed_dt", [False, True])
def test_local_slabs_equal_the_single_process_step_bitwise(nslabs, fixed_dt):
    w = workload(fixed_dt)
    nsteps = 3
    f0 = I.initial_condition(w, np.float64)
    nx = w.n[0] // nslabs
    slabs = [OracleSlab(w, r * nx, nx, f0) for r in range(nslabs)]
    step = ShardedStep(slabs, LocalExchange())
    if fixed_dt:
        assert step.nghost(step.dt) == 4
    t = step.step(nsteps)
    got = np.concatenate([s.f for s in slabs])
    ref = reference(w, nsteps)
    assert t == ref.t
    assert np.array_equal(got, ref.f)


def test_slabs_thinner_than_the_halo_are_refused():
    w = workload(fixed_dt=True)                 # four ghost planes
    f0 = I.initial_condition(w, np.float64)
    slabs = [OracleSlab(w, r * 3, 3, f0) for r in range(4)]
    step = ShardedStep(slabs, LocalExchange())
    with pytest.raises(ValueError):
        step.step(1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, fixed_dt, nsteps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = workload(fixed_dt)
        f0 = I.initial_condition(w, np.float64)
        nx = w.n[0] // world
        slab = OracleSlab(w, rank * nx, nx, f0)
        step = ShardedStep([slab], DistExchange())
        t = step.step(nsteps)
        out[rank] = (t, slab.f.copy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,fixed_dt", [(2, False), (3, True)])
@pytest.mark.skipif(torch.cuda.is_available(), reason="CPU gloo check")
def test_gloo_ranks_equal_the_single_process_step_bitwise(world, fixed_dt):
    """One slab per gloo rank: the halo planes travel point to point (with
    two ranks both neighbours are the same peer), the line maxima by
    all-reduce, the density by all-gather."""
    import torch.multiprocessing as mp
    nsteps = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), fixed_dt, nsteps, out), nprocs=world, join=True)
    w = workload(fixed_dt)
    ref = reference(w, nsteps)
    got = np.concatenate([out[r][1] for r in range(world)])
    assert all(out[r][0] == ref.t for r in range(world))
    assert np.array_equal(got, ref.f)
