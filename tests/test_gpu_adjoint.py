"""GPU discrete adjoint against the FP64 oracle's adjoint (same frozen-branch
rules) and against central finite differences of the GPU forward map."""
import gc
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


def gpu_sim(w, f_np, dtype=None):
    from paper_1206_6152_gb300.vlasov import VlasovPoisson, config_of
    tdt = dtype or (torch.float32 if w.dtype == "f32" else torch.float64)
    f = torch.from_numpy(np.ascontiguousarray(f_np)).to(DEV, tdt)
    return VlasovPoisson(config_of(w, tdt), f), f


@pytest.mark.gpu
@pytest.mark.parametrize("space_bc", ["periodic", "outflow"])
def test_sweep_adjoint_matches_oracle(space_bc):
    w = I.small_maxwell(n=(6, 5, 4), nv=(8, 7, 6), dtype="f64", amp=0.3, space_bc=space_bc)
    grid = O.Grid.of(w)
    rng = np.random.default_rng(21)
    f0 = I.initial_condition(w) * (1 + 0.5 * rng.random(w.shape))     # tie free
    acc = rng.normal(size=(3,) + w.n) * 3
    sim, f = gpu_sim(w, f0)
    sim.set_accel(torch.from_numpy(acc))
    per = space_bc == "periodic"
    for axis in range(6):
        for tau in (0.017, -0.023, 0.31):
            lam0 = rng.normal(size=w.shape)
            fin = torch.from_numpy(f0).to(DEV)
            lam = torch.from_numpy(lam0).to(DEV)
            lg = torch.zeros((3,) + w.n, dtype=torch.float64, device=DEV)
            sim.sweep_adjoint(axis, tau, fin, lam, lg)
            ref = lam0.copy()
            ds = np.zeros(int(np.prod(w.n)))
            if axis < 3:
                O.sweep_adjoint(f0, ref, axis, grid.vc(axis), tau, grid.dx[axis], per, None)
            else:
                O.sweep_adjoint(f0, ref, axis, acc[axis - 3], tau, grid.dv[axis - 3], False, ds)
            got = lam.cpu().numpy()
            assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), (axis, tau)
            if axis >= 3:
                gg = lg.cpu().numpy()[axis - 3].reshape(-1)
                assert np.abs(gg - ds).max() <= 1e-10 * max(np.abs(ds).max(), 1e-300), (axis, tau)
    sim.close()


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,shape,space_bc", [
    ("f64", dict(n=(16, 16, 16), nv=(16, 16, 16)), "periodic"),
    ("f32", dict(n=(16, 32, 16), nv=(16, 16, 32)), "periodic"),
    ("f32", dict(n=(16, 32, 16), nv=(16, 16, 32)), "outflow"),
    ("f32", dict(n=(4, 2, 2), nv=(32, 32, 32)), "periodic"),
    ("f32", dict(n=(4, 4, 2), nv=(16, 16, 16)), "periodic"),
    ("f32", dict(n=(48, 2, 2), nv=(2, 4, 6)), "periodic"),
    ("f32", dict(n=(48, 2, 2), nv=(2, 4, 6)), "outflow"),
    ("f32", dict(n=(2, 2, 1), nv=(48, 48, 48)), "periodic"),
])
def test_register_adjoint_sweeps_match_oracle(dtype, shape, space_bc):
    """Line lengths served by the register-line adjoint kernels: FP64 lines
    of 16; FP32 packed line pairs of 16 and 32 along position axes (both
    boundary kinds, and pairs of z lines with different speeds) and along vx
    and vy of 16^3 and 32^3 cubes, and the warp-staged vz rows; the same for
    lines of 48 (x lines, 48^3 cubes)."""
    w = I.small_maxwell(dtype=dtype, amp=0.3, space_bc=space_bc, **shape)
    w = w.replace(box_lo=(-0.5,) * 3, box_hi=(0.5,) * 3)
    grid = O.Grid.of(w)
    rng = np.random.default_rng(9)
    npdt = np.float32 if dtype == "f32" else np.float64
    f0 = (I.initial_condition(w, np.float64) * (1 + 0.5 * rng.random(w.shape))).astype(npdt)
    acc = rng.normal(size=(3,) + w.n) * 3
    sim, f = gpu_sim(w, f0)
    sim.set_accel(torch.from_numpy(acc))
    for axis in range(6):
        for tau in (0.011, -0.017):
            lam0 = rng.normal(size=w.shape).astype(npdt)
            lam = torch.from_numpy(lam0).to(DEV)
            lg = torch.zeros((3,) + w.n, dtype=torch.float64, device=DEV)
            sim.sweep_adjoint(axis, tau, torch.from_numpy(f0).to(DEV), lam, lg)
            ref = lam0.astype(np.float64)
            ds = np.zeros(int(np.prod(w.n)))
            f64 = f0.astype(np.float64)
            if axis < 3:
                O.sweep_adjoint(f64, ref, axis, grid.vc(axis), tau, grid.dx[axis],
                                space_bc == "periodic", None)
            else:
                O.sweep_adjoint(f64, ref, axis, acc[axis - 3], tau, grid.dv[axis - 3], False, ds)
            got = lam.cpu().numpy().astype(np.float64)
            rel = np.abs(got - ref).sum() / np.abs(ref).sum()
            assert rel <= (1e-13 if dtype == "f64" else 1e-6), (axis, tau, rel)
            if axis >= 3:
                gg = lg.cpu().numpy()[axis - 3].reshape(-1)
                relg = np.abs(gg - ds).sum() / np.abs(ds).sum()
                assert relg <= (1e-12 if dtype == "f64" else 1e-5), (axis, tau, relg)
    sim.close()


@pytest.mark.gpu
@pytest.mark.parametrize("states", [0, 1, 3])
@pytest.mark.parametrize("bc", ["periodic", "isolated"])
def test_adjoint_step_matches_oracle(bc, states):
    w = I.small_maxwell(n=(6, 5, 4), nv=(8, 7, 6), dtype="f64", amp=0.2, G=20.0)
    w = w.replace(dt_fixed=0.01)
    if bc == "isolated":
        w = w.replace(box_lo=(-0.3, -0.25, -0.2), box_hi=(0.3, 0.25, 0.2), poisson_bc="isolated",
                      space_bc="outflow")
    grid = O.Grid.of(w)
    rng = np.random.default_rng(3)
    f0 = I.initial_condition(w) * (1 + 0.2 * rng.random(w.shape))
    sim, f = gpu_sim(w, f0)
    sim.set_adjoint_states(states)           # 1, 3: inputs recomputed with two or three states
    g0 = sim.field()[2]
    lam_f = torch.from_numpy(rng.normal(size=w.shape)).to(DEV)
    lam_g = torch.from_numpy(rng.normal(size=(3,) + w.n)).to(DEV)
    lf0, lg0 = lam_f.cpu().numpy(), lam_g.cpu().numpy()
    sim.adjoint_step(torch.from_numpy(f0).to(DEV), g0, lam_f, lam_g)
    osim = O.Simulation(f0, grid, O.Params.of(w))
    rf, rg = O.adjoint_step(osim, f0, osim.g, lf0, lg0)
    assert np.abs(g0.cpu().numpy() - osim.g).max() <= 1e-11 * np.abs(osim.g).max()
    got_f, got_g = lam_f.cpu().numpy(), lam_g.cpu().numpy()
    assert np.abs(got_f - rf).max() <= 1e-9 * np.abs(rf).max()
    assert np.abs(got_g - rg).max() <= 1e-9 * np.abs(rg).max()
    sim.close()


@pytest.mark.gpu
@pytest.mark.parametrize("G,n,states", [(20.0, (16, 2, 2), 0), (200.0, (16, 2, 2), 0),
                                        (20.0, (2, 16, 16), 0), (20.0, (16, 2, 2), 1),
                                        (2000.0, (2, 16, 16), 1), (20.0, (16, 2, 2), 3),
                                        (20.0, (2, 16, 16), 3)])
def test_adjoint_step_fp32_register_kernels_match_oracle(G, n, states):
    """FP32 adjoint step on grids served by the packed kernels against the
    FP64 oracle's adjoint step: x lines of 16 with the density broadcast
    added on load, 16^3 velocity cubes (vz input recomputed); y and z lines
    of 16 (the replay's fused z + y drift keeping the z output, the z
    adjoint's warp-uniform direction map, pairs straddling v_z = 0).  With
    the large G the kicks shift by whole cells: the replay's shifted-cube
    path and the adjoint's fix-up pass."""
    w = I.small_maxwell(n=n, nv=(16, 16, 16), dtype="f32", amp=0.2, G=G)
    half = tuple(0.5 if m == 16 else 0.05 for m in n)
    w = w.replace(dt_fixed=0.01, box_lo=tuple(-h for h in half), box_hi=half)
    grid = O.Grid.of(w)
    rng = np.random.default_rng(4)
    f0 = (I.initial_condition(w, np.float64) * (1 + 0.2 * rng.random(w.shape))).astype(np.float32)
    sim, f = gpu_sim(w, f0)
    sim.set_adjoint_states(states)
    g0 = sim.field()[2]
    lam_f = torch.from_numpy(rng.normal(size=w.shape).astype(np.float32)).to(DEV)
    lam_g = torch.from_numpy(rng.normal(size=(3,) + w.n)).to(DEV)
    lf0, lg0 = lam_f.cpu().numpy().astype(np.float64), lam_g.cpu().numpy()
    m_out = sim.energy()["M_out"]
    sim.adjoint_step(torch.from_numpy(f0).to(DEV), g0, lam_f, lam_g)
    assert sim.energy()["M_out"] == m_out        # the replay's outflow is not the run's
    f64 = f0.astype(np.float64)
    osim = O.Simulation(f64, grid, O.Params.of(w))
    rf, rg = O.adjoint_step(osim, f64, osim.g, lf0, lg0)
    got_f, got_g = lam_f.cpu().numpy().astype(np.float64), lam_g.cpu().numpy()
    if G > 100:
        assert np.abs(osim.g).max() * 0.5 * w.dt_fixed / grid.dv[0] > 1.5   # whole-cell kicks
    assert np.abs(got_f - rf).sum() / np.abs(rf).sum() <= 2e-5
    assert np.abs(got_g - rg).sum() / np.abs(rg).sum() <= 2e-5
    sim.close()


@pytest.mark.gpu
@pytest.mark.parametrize("states", [0, 1, 3])
def test_adjoint_step_48_cubes_match_oracle(states):
    """FP32 adjoint step with 48^3 velocity cubes (out-of-place replay kicks,
    per-axis register adjoints over any number of cubes) against the FP64
    oracle, with nine kept states, with two and with three."""
    w = I.large_c5().replace(n=(2, 2, 2), box_lo=(-0.5,) * 3, box_hi=(0.5,) * 3, G=40.0,
                             dt_fixed=0.01)
    grid = O.Grid.of(w)
    rng = np.random.default_rng(8)
    f0 = (I.initial_condition(w, np.float64) * (1 + 0.2 * rng.random(w.shape))).astype(np.float32)
    sim, f = gpu_sim(w, f0)
    sim.set_adjoint_states(states)
    g0 = sim.field()[2]
    lam_f = torch.from_numpy(rng.normal(size=w.shape).astype(np.float32)).to(DEV)
    lam_g = torch.from_numpy(rng.normal(size=(3,) + w.n)).to(DEV)
    lf0, lg0 = lam_f.cpu().numpy().astype(np.float64), lam_g.cpu().numpy()
    sim.adjoint_step(torch.from_numpy(f0).to(DEV), g0, lam_f, lam_g)
    f64 = f0.astype(np.float64)
    osim = O.Simulation(f64, grid, O.Params.of(w))
    rf, rg = O.adjoint_step(osim, f64, osim.g, lf0, lg0)
    got_f, got_g = lam_f.cpu().numpy().astype(np.float64), lam_g.cpu().numpy()
    assert np.abs(got_f - rf).sum() / np.abs(rf).sum() <= 2e-5
    assert np.abs(got_g - rg).sum() / np.abs(rg).sum() <= 2e-5
    sim.close()


@pytest.mark.gpu
@pytest.mark.parametrize("nx", [16, 32, 48])
def test_adjoint_step_fp32_x_lines_match_oracle(nx):
    """FP32 adjoint step on x lines of 16, 32 and 48 (the line-pair x-drift
    adjoint with the density cotangent added as it loads the cotangent)
    against the oracle's adjoint step.  The outer v_x cells shift by 1.44
    cells: the pair kernel leaves those lines to the fix-up sweep, which must
    see their density cotangent too."""
    w = I.small_maxwell(n=(nx, 2, 2), nv=(4, 4, 6), dtype="f32", amp=0.3, G=20.0)
    w = w.replace(box_lo=(-0.5, -0.05, -0.05), box_hi=(0.5, 0.05, 0.05), dt_fixed=0.48 / nx)
    rng = np.random.default_rng(12)
    f0 = (I.initial_condition(w, np.float64) * (1 + 0.2 * rng.random(w.shape))).astype(np.float32)
    sim, f = gpu_sim(w, f0)
    g0 = sim.field()[2]
    lam_f = torch.from_numpy(rng.normal(size=w.shape).astype(np.float32)).to(DEV)
    lam_g = torch.from_numpy(rng.normal(size=(3,) + w.n)).to(DEV)
    lf0, lg0 = lam_f.cpu().numpy().astype(np.float64), lam_g.cpu().numpy()
    sim.adjoint_step(torch.from_numpy(f0).to(DEV), g0, lam_f, lam_g)
    f64 = f0.astype(np.float64)
    osim = O.Simulation(f64, O.Grid.of(w), O.Params.of(w))
    rf, rg = O.adjoint_step(osim, f64, osim.g, lf0, lg0)
    got_f, got_g = lam_f.cpu().numpy().astype(np.float64), lam_g.cpu().numpy()
    assert np.abs(got_f - rf).sum() / np.abs(rf).sum() <= 2e-5
    assert np.abs(got_g - rg).sum() / np.abs(rg).sum() <= 2e-5
    sim.close()


def _mode_f0(w, amps, dtype):
    """f0(A) = rho_bar (1 + sum_m A_m cos(k_m.x + th_m)) M(v), in torch."""
    fields = torch.from_numpy(I.mode_fields(w)).to(DEV)
    mv = torch.from_numpy(I.maxwellian_v(w)).to(DEV)
    rho = w.rho_bar * (1 + torch.tensordot(amps.to(torch.float64), fields, dims=1))
    return (rho[..., None, None, None] * mv).to(dtype).contiguous()


def _J_of(sim, f0, nsteps, kind, target):
    with torch.no_grad():
        sim.f.copy_(f0)
        sim.refresh_field()
        sim.step(nsteps)
        lam = torch.empty_like(sim.f)
        return sim.functional(kind, lam, target)


@pytest.mark.gpu
@pytest.mark.parametrize("kind,keep", [(0, None), (1, None), (0, False)])
def test_trajectory_gradient_fp64_matches_fd(kind, keep):
    from paper_1206_6152_gb300.adjoint import trajectory_functional
    w = I.small_maxwell(n=(8, 6, 5), nv=(10, 8, 9), dtype="f64", amp=0.1, G=25.0)
    w = w.replace(dt_fixed=0.008)
    amps0 = torch.tensor([m[1] for m in w.modes], dtype=torch.float64, device=DEV)
    sim, f = gpu_sim(w, np.zeros(w.shape))
    target = None
    if kind == 1:
        target = torch.from_numpy(w.rho_bar * (1 + 0.05 * I.mode_fields(w)[0])).to(DEV)
    nsteps = 6
    amps = amps0.clone().requires_grad_(True)
    J = trajectory_functional(_mode_f0(w, amps, torch.float64), sim, nsteps, every=4, kind=kind,
                              target=target, keep_states=keep)
    J.backward()
    grad = amps.grad.cpu().numpy()
    for m in range(len(w.modes)):
        h = 1e-7
        ap, am = amps0.clone(), amps0.clone()
        ap[m] += h
        am[m] -= h
        fd = (_J_of(sim, _mode_f0(w, ap, torch.float64), nsteps, kind, target)
              - _J_of(sim, _mode_f0(w, am, torch.float64), nsteps, kind, target)) / (2 * h)
        assert grad[m] == pytest.approx(fd, rel=1e-5, abs=1e-9 * abs(J.item())), m
    sim.close()


@pytest.mark.gpu
@pytest.mark.slow
def test_jeans32_modes3_gradient_fp32_matches_fd():
    """The 32^3 x 32^3 FP32 Jeans box with 3 seeded modes: gradient of the
    final field energy w.r.t. the mode amplitudes through the adjoint with
    checkpoints every 10 steps, against central differences.  In the linear
    regime J is quadratic in the amplitudes, so a central difference is exact
    for any step; the step (10% of each amplitude) keeps the FP32 rounding of
    J below the difference.  The Landau-damped mode (k/k_J = 1.5) has, after
    100 steps, a gradient ~250 times smaller than the growing ones, below the
    FP32 resolution of a difference quotient of J; errors are therefore
    measured against the largest gradient component."""
    from paper_1206_6152_gb300.adjoint import trajectory_functional
    w = I.adjoint_c4()
    nsteps = w.steps                     # 100 steps, checkpoints every 10
    amps0 = torch.tensor([m[1] for m in w.modes], dtype=torch.float64, device=DEV)
    sim, f = gpu_sim(w, np.zeros(w.shape, np.float32))
    amps = amps0.clone().requires_grad_(True)
    J = trajectory_functional(_mode_f0(w, amps, torch.float32), sim, nsteps, every=10, kind=0)
    J.backward()
    grad = amps.grad.cpu().numpy()
    fds = []
    for m in range(len(w.modes)):
        h = 0.1 * float(amps0[m])
        ap, am = amps0.clone(), amps0.clone()
        ap[m] += h
        am[m] -= h
        fds.append((_J_of(sim, _mode_f0(w, ap, torch.float32), nsteps, 0, None)
                    - _J_of(sim, _mode_f0(w, am, torch.float32), nsteps, 0, None)) / (2 * h))
    fds = np.array(fds)
    assert np.abs(grad - fds).max() <= 1e-3 * np.abs(fds).max(), (grad, fds)
    # directional derivative along the amplitude vector itself
    eps = 0.05
    fd = (_J_of(sim, _mode_f0(w, amps0 * (1 + eps), torch.float32), nsteps, 0, None)
          - _J_of(sim, _mode_f0(w, amps0 * (1 - eps), torch.float32), nsteps, 0, None)) / (2 * eps)
    assert float(np.dot(grad, amps0.cpu().numpy())) == pytest.approx(fd, rel=1e-3)
    sim.close()


def _fill_mode_f0(w, amps, out):
    """out <- f0(A) = rho_bar (1 + sum_m A_m cos(k_m.x + th_m)) M(v) in FP64,
    rounded once to out's dtype, in chunks of positions (a 49 GB f has no
    room for an FP64 copy)."""
    fields = torch.from_numpy(I.mode_fields(w).reshape(len(w.modes), -1)).to(DEV)
    rho = w.rho_bar * (1 + torch.as_tensor(list(amps), dtype=torch.float64, device=DEV) @ fields)
    mv = torch.from_numpy(I.maxwellian_v(w).reshape(-1)).to(DEV)
    o = out.view(rho.numel(), -1)
    step = max(1, (1 << 26) // mv.numel())
    for s in range(0, rho.numel(), step):
        o[s:s + step] = (rho[s:s + step, None] * mv[None, :]).to(out.dtype)
    return out


@pytest.mark.gpu
@pytest.mark.slow
def test_jeans48_modes8_trajectory_gradient_matches_fd():
    """The 48^3 x 48^3 FP32 forward+adjoint workload at a reduced step count:
    20 steps from f0(A) with checkpoints every 10 (two checkpoints; they go
    to pinned host memory because the device cannot hold them beside f, f0,
    the cotangent and the adjoint's scratch states, two here) and every step-start
    state recomputed from its checkpoint.  The gradient of the final field
    energy with respect to the eight mode amplitudes, dJ/dA_m = rho_bar
    sum_x cos(k_m.x + th_m) sum_v lambda_0(x, v) M(v) with lambda_0 = dJ/df0
    per cell, against central differences (1% of each amplitude; J is
    quadratic in A in the linear regime), errors against the largest
    component, and along the amplitude vector itself."""
    from paper_1206_6152_gb300.adjoint import trajectory_functional
    from paper_1206_6152_gb300.vlasov import VlasovPoisson, config_of
    w = I.large_c5()
    nsteps, every = 20, 10
    amps0 = np.array([m[1] for m in w.modes])
    gc.collect()
    torch.cuda.empty_cache()
    f = torch.zeros(w.shape, dtype=torch.float32, device=DEV)
    sim = VlasovPoisson(config_of(w), f)
    f0 = _fill_mode_f0(w, amps0, torch.empty_like(f)).requires_grad_(True)
    J = trajectory_functional(f0, sim, nsteps, every=every, kind=0, keep_states=False)
    J.backward()
    lam0 = f0.grad
    mv = torch.from_numpy(I.maxwellian_v(w).reshape(-1)).to(DEV)
    npos = int(np.prod(w.n))
    s = torch.empty(npos, dtype=torch.float64, device=DEV)
    lv = lam0.view(npos, -1)
    for a in range(0, npos, 2304):
        s[a:a + 2304] = lv[a:a + 2304].double() @ mv
    fields = torch.from_numpy(I.mode_fields(w).reshape(len(w.modes), -1)).to(DEV)
    grad = (w.rho_bar * (fields @ s)).cpu().numpy()
    del f0, lam0, lv, J
    torch.cuda.empty_cache()

    lam = torch.empty_like(f)

    def J_of(amps):
        with torch.no_grad():
            _fill_mode_f0(w, amps, sim.f)
            sim.refresh_field()
            sim.step(nsteps)
            return sim.functional(0, lam)

    fds = []
    for m in range(len(amps0)):
        h = 0.01 * amps0[m]
        ap, am = amps0.copy(), amps0.copy()
        ap[m] += h
        am[m] -= h
        fds.append((J_of(ap) - J_of(am)) / (2 * h))
    fds = np.array(fds)
    assert np.abs(grad - fds).max() <= 1e-3 * np.abs(fds).max(), (grad, fds)
    eps = 0.01
    fd = (J_of(amps0 * (1 + eps)) - J_of(amps0 * (1 - eps))) / (2 * eps)
    assert float(np.dot(grad, amps0)) == pytest.approx(fd, rel=1e-3)
    sim.close()
