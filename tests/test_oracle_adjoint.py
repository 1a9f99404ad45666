"""Pins of the oracle's discrete adjoint (not in the paper) against central
finite differences of the oracle's own forward map, which is pinned to the
paper elsewhere.  Away from limiter kinks the frozen-branch adjoint is the
exact derivative, so the agreement is limited only by the FD truncation."""
import numpy as np
import pytest

from oracle import vp_oracle as O
from paper_1206_6152_gb300 import inputs as I


def limiter_arms(f, alpha, periodic):
    """The branch pattern of one line update, restated on the test side from
    the corrector's case split (Filbet et al. 2001, ratio form): for every
    cell of the line in upwind order, which arm each corrected difference
    takes (0: unlimited, 1: limited by the positivity bound, 2: limited by
    the maximum bound), and the first position of the line maximum.  A
    central difference is a valid check of the frozen-branch adjoint only if
    both of its runs keep the pattern of the unperturbed line."""
    g = np.asarray(f, dtype=np.float64)[::-1] if alpha < 0 else np.asarray(f, dtype=np.float64)
    n = g.size
    finf = max(float(g.max()), 0.0)

    def cell(j):
        if periodic:
            return g[j % n]
        return g[j] if 0 <= j < n else 0.0

    pattern = []
    for j in range(n):
        fm, f0, fp = cell(j - 1), cell(j), cell(j + 1)
        dp, dm = fp - f0, f0 - fm
        ap = 1 if dp > 0 and 2 * f0 < dp else (2 if dp < 0 and 2 * (finf - f0) < -dp else 0)
        am = 2 if dm > 0 and 2 * (finf - f0) < dm else (1 if dm < 0 and 2 * f0 < -dm else 0)
        pattern.append((ap, am))
    return pattern, int(np.argmax(g))


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("alpha", [0.23, 0.81, 1.37, -0.44, -2.61])
def test_line_adjoint_matches_fd(periodic, alpha):
    rng = np.random.default_rng(4)
    n = 11
    f = rng.random(n) + 0.05
    f[3] = 0.0                         # a zero cell exercises the limiter
    w = rng.normal(size=n)
    lam, dalpha = O.pfc_line_adjoint(f, w, alpha, periodic)
    h = 1e-7
    arms = limiter_arms(f, alpha, periodic)
    assert any(a != (0, 0) for a in arms[0])      # the line exercises the corrector
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        if f[j] == 0.0:                # one-sided: f >= 0
            assert limiter_arms(f + e, alpha, periodic) == arms
            fd = (w @ O.pfc_line(f + e, alpha, periodic) - w @ O.pfc_line(f, alpha, periodic)) / h
            assert lam[j] == pytest.approx(fd, rel=1e-5, abs=1e-6)
            continue
        assert limiter_arms(f + e, alpha, periodic) == arms == limiter_arms(f - e, alpha, periodic)
        fd = (w @ O.pfc_line(f + e, alpha, periodic) - w @ O.pfc_line(f - e, alpha, periodic)) / (2 * h)
        assert lam[j] == pytest.approx(fd, rel=1e-6, abs=1e-7)
    fd = (w @ O.pfc_line(f, alpha + h, periodic) - w @ O.pfc_line(f, alpha - h, periodic)) / (2 * h)
    assert dalpha == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_sweep_adjoint_dot_products():
    w = I.small_maxwell(n=(4, 3, 5), nv=(6, 5, 7), amp=0.3)
    grid = O.Grid.of(w)
    rng = np.random.default_rng(5)
    # random data: no ties at the line maxima, so the map is smooth here
    f0 = I.initial_condition(w) * (1 + 0.5 * rng.random(w.shape))
    acc = rng.normal(size=(3,) + w.n) * 3
    for axis in range(6):
        if axis < 3:
            speed, tau, h, per = grid.vc(axis), 0.021, grid.dx[axis], True
        else:
            speed, tau, h, per = acc[axis - 3], 0.07, grid.dv[axis - 3], False
        wt = rng.normal(size=w.shape)
        lam = wt.copy()
        ds = np.zeros(speed.size)
        O.sweep_adjoint(f0, lam, axis, speed, tau, h, per, ds)
        d = rng.normal(size=w.shape) * f0           # relative perturbation
        # the frozen-branch map is linear, so central FD is exact except
        # where +-eps crosses a limiter threshold somewhere in the array;
        # such crossings shift the FD by ~1e-6 relative at this eps
        eps = 1e-7

        def J(f, sp=speed):
            g = f.copy()
            O.sweep(g, axis, sp, tau, h, per)
            return float(np.sum(wt * g))

        fd = (J(f0 + eps * d) - J(f0 - eps * d)) / (2 * eps)
        assert float(np.sum(lam * d)) == pytest.approx(fd, rel=1e-5)
        ds_dir = rng.normal(size=speed.shape)
        fd = (J(f0, speed + eps * ds_dir) - J(f0, speed - eps * ds_dir)) / (2 * eps)
        assert float(np.sum(ds.reshape(speed.shape) * ds_dir)) == pytest.approx(fd, rel=1e-5)


def _forward_J(w, amps, nsteps, functional, target=None):
    grid = O.Grid.of(w)
    f0 = I.initial_condition(w, np.float64, amplitudes=amps)
    sim = O.Simulation(f0, grid, O.Params.of(w))
    sim.step(nsteps)
    if functional == "U":
        return O.field_energy_gradient(sim.f, sim)[0]
    return O.density_misfit_gradient(sim.f, sim, target)[0]


def _adjoint_grad(w, nsteps, functional, target=None):
    grid = O.Grid.of(w)
    f0 = I.initial_condition(w, np.float64)
    sim = O.Simulation(f0, grid, O.Params.of(w))
    states = []
    for _ in range(nsteps):
        states.append((sim.f.copy(), sim.g.copy()))
        sim.step()
    if functional == "U":
        J, lam_f = O.field_energy_gradient(sim.f, sim)
    else:
        J, lam_f = O.density_misfit_gradient(sim.f, sim, target)
    lam_g = np.zeros_like(sim.g)
    for fn, gn in reversed(states):
        lam_f, lam_g = O.adjoint_step(sim, fn, gn, lam_f, lam_g)
    lam_f0 = lam_f + O.field_adjoint(lam_g, sim)
    return J, lam_f0


@pytest.mark.parametrize("functional", ["U", "misfit"])
def test_step_adjoint_matches_fd_in_mode_amplitudes(functional):
    w = I.small_maxwell(n=(6, 5, 4), nv=(8, 7, 6), amp=0.1, G=20.0)
    w = w.replace(dt_fixed=0.01)
    nsteps = 2
    target = None
    if functional == "misfit":
        target = w.rho_bar * (1 + 0.05 * I.mode_fields(w)[0])
    J, lam_f0 = _adjoint_grad(w, nsteps, functional, target)
    mv = I.maxwellian_v(w)
    fields = I.mode_fields(w)
    amps = np.array([m[1] for m in w.modes])
    for m in range(len(w.modes)):
        grad = float(np.sum(lam_f0 * (w.rho_bar * fields[m])[..., None, None, None] * mv))
        h = 1e-7          # small enough that no limiter threshold is crossed
        ap, am = amps.copy(), amps.copy()
        ap[m] += h
        am[m] -= h
        fd = (_forward_J(w, ap, nsteps, functional, target)
              - _forward_J(w, am, nsteps, functional, target)) / (2 * h)
        assert grad == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(J))
