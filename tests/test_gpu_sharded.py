"""The library's pieces of the x-slab decomposition (Sec. 2.3) on one GPU:
slab contexts with the ghosted x drift, the per-line maxima along x and a
field-only context per slab, driven by sharded.ShardedStep with the slabs
exchanging by direct copies in one process (the kernels of different slabs
never wait on each other).  The slabs' split steps against the single-context
step of the same box and against the FP64 oracle; argument and state
checks of the new entry points."""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = pytest.mark.skip(reason="needs a CUDA GPU")

from oracle import vp_oracle as O  # noqa: E402
from paper_1206_6152_gb300 import inputs as I  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1206_6152_gb300 import build as B
    B.build()


def workload(dtype, fixed_dt=False):
    w = I.small_maxwell(n=(12, 4, 5), nv=(6, 4, 5), dtype=dtype, amp=0.3, G=25.0)
    w = w.replace(box_lo=(-0.5, -0.2, -0.25), box_hi=(0.5, 0.2, 0.25))
    if fixed_dt:
        dv = (w.vhi[0] - w.vlo[0]) / 6
        vmax = max(abs(w.vlo[0] + 0.5 * dv), abs(w.vhi[0] - 0.5 * dv))
        w = w.replace(dt_fixed=2.6 * (1.0 / 12) / vmax)      # x shifts up to 2.6 cells
    return w


@pytest.mark.gpu
@pytest.mark.parametrize("nslabs", [1, 2, 3])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("fixed_dt", [False, True])
def test_slabs_equal_the_whole_box(nslabs, dtype, tol, fixed_dt):
    from paper_1206_6152_gb300.sharded import LibrarySlab, LocalExchange, ShardedStep
    from paper_1206_6152_gb300.vlasov import VlasovPoisson, config_of
    w = workload(dtype, fixed_dt)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    f0 = I.initial_condition(w)
    nsteps = 3
    # the whole box in one context
    fw = torch.from_numpy(f0).to(DEV, tdt)
    with VlasovPoisson(config_of(w, tdt), fw) as sim:
        t_whole = sim.step(nsteps, sync=True)
    whole = fw.cpu().numpy().astype(np.float64)
    # the same box as slabs of one tensor
    fs = torch.from_numpy(f0).to(DEV, tdt)
    nx = w.n[0] // nslabs
    cfg = config_of(w, tdt)
    slabs = [LibrarySlab(cfg, r * nx, fs[r * nx:(r + 1) * nx]) for r in range(nslabs)]
    try:
        step = ShardedStep(slabs, LocalExchange())
        if fixed_dt:
            assert step.nghost(step.dt) == 4
        t = step.step(nsteps)
        torch.cuda.synchronize()
        got = fs.cpu().numpy().astype(np.float64)
    finally:
        for s in slabs:
            s.close()
    assert t == pytest.approx(t_whole, rel=1e-13 if dtype == "f64" else 1e-6)
    assert np.abs(got - whole).sum() / np.abs(whole).sum() <= tol
    assert got.min() >= 0.0
    if dtype == "f64":
        ref = O.Simulation(f0, O.Grid.of(w), O.Params.of(w))
        ref.step(nsteps)
        assert np.abs(got - ref.f).sum() / np.abs(ref.f).sum() <= 1e-11


@pytest.mark.gpu
@pytest.mark.parametrize("nslabs", [2, 4])
def test_slabs_on_the_register_kernels(nslabs):
    """FP32 slabs whose kicks run as the fused one-pass kick of 16^3 cubes
    (K2 of a step and K1 of the next together) and whose z and y drifts run
    as the fused drift (N_y = N_z = 32): the slabs' steps against the whole
    box's vp_step and against the FP64 oracle."""
    from paper_1206_6152_gb300.sharded import LibrarySlab, LocalExchange, ShardedStep
    from paper_1206_6152_gb300.vlasov import VlasovPoisson, config_of
    w = I.small_maxwell(n=(8, 32, 32), nv=(16, 16, 16), dtype="f32", amp=0.3, G=25.0)
    w = w.replace(box_lo=(-0.5,) * 3, box_hi=(0.5,) * 3)
    f0 = I.initial_condition(w)
    nsteps = 3
    fw = torch.from_numpy(f0).to(DEV, torch.float32)
    with VlasovPoisson(config_of(w), fw) as sim:
        t_whole = sim.step(nsteps, sync=True)
    whole = fw.cpu().numpy().astype(np.float64)
    fs = torch.from_numpy(f0).to(DEV, torch.float32)
    nx = w.n[0] // nslabs
    cfg = config_of(w)
    slabs = [LibrarySlab(cfg, r * nx, fs[r * nx:(r + 1) * nx]) for r in range(nslabs)]
    try:
        t = ShardedStep(slabs, LocalExchange()).step(nsteps)
        torch.cuda.synchronize()
        got = fs.cpu().numpy().astype(np.float64)
    finally:
        for s in slabs:
            s.close()
    assert t == pytest.approx(t_whole, rel=1e-6)
    assert np.abs(got - whole).sum() / np.abs(whole).sum() <= 1e-5
    ref = O.Simulation(f0.astype(np.float64), O.Grid.of(w), O.Params.of(w))
    ref.step(nsteps)
    assert np.abs(got - ref.f).sum() / np.abs(ref.f).sum() <= 1e-5
    assert got.min() >= 0.0


@pytest.mark.gpu
def test_slab_entry_points_check_their_arguments():
    from paper_1206_6152_gb300 import _lib
    from paper_1206_6152_gb300.sharded import LibrarySlab
    from paper_1206_6152_gb300.vlasov import config_of
    lib = _lib.load()
    w = workload("f64", fixed_dt=True)
    f = torch.from_numpy(I.initial_condition(w)).to(DEV)
    slab = LibrarySlab(config_of(w, torch.float64), 0, f[0:6])
    try:
        lm = slab.line_max_x()
        assert torch.equal(lm, torch.clamp(f[0:6].max(dim=0).values, min=0.0))
        plane = torch.zeros((3,) + tuple(f.shape[1:]), dtype=f.dtype, device=DEV)
        # x shifts of up to 2.6 cells need four ghost planes: three are refused
        rc = lib.vp_drift_x_ghosted(slab.sim._ctx, float(w.dt_fixed), ctypes.c_void_p(plane.data_ptr()),
                                    ctypes.c_void_p(plane.data_ptr()), 3, ctypes.c_void_p(lm.data_ptr()))
        assert rc == -5
        # a field-only context has no f
        rc = lib.vp_step(slab._fctx, 1, None)
        assert rc == -6
        rc = lib.vp_line_max_x(slab._fctx, ctypes.c_void_p(lm.data_ptr()))
        assert rc == -6
        assert lib.vp_kick(slab._fctx, 0.01, 0.0) == -6
        assert lib.vp_drift_yz(slab._fctx, 0.01) == -6
        # non-finite durations are refused
        assert lib.vp_kick(slab.sim._ctx, math.nan, 0.0) == -5
        assert lib.vp_kick(slab.sim._ctx, 0.01, math.inf) == -5
        assert lib.vp_drift_yz(slab.sim._ctx, math.nan) == -5
        # its field is the oracle's
        rho = slab.density()
        rho_all = torch.cat([rho, rho])
        g, dt = slab.field(rho_all)
        grid = O.Grid.of(w)
        phi = O.poisson(rho_all.cpu().numpy(), grid, w.G, "periodic")
        g_o = O.force(phi, grid, "periodic")
        assert np.abs(g.cpu().numpy() - g_o).max() <= 1e-11 * np.abs(g_o).max()
        assert dt == w.dt_fixed
    finally:
        slab.close()
