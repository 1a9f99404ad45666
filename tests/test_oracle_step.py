"""Pins of the oracle's 6D sweeps and split step (Sec. 2.1, Eq. integration)
and of its physics against the linear theory of Sec. 3.2 (Eq. dispersion)
and the conservation figures the paper quotes for Tests 1 and 2."""
import math

import numpy as np
import pytest

from conftest import golden
from scipy.optimize import brentq
from scipy.special import erfcx, erf

from oracle import vp_oracle as O
from paper_1206_6152_gb300 import inputs as I


def test_sweep_walks_every_line_with_its_speed():
    w = I.small_maxwell(n=(4, 3, 5), nv=(6, 5, 4))
    grid = O.Grid.of(w)
    rng = np.random.default_rng(0)
    f0 = rng.random(w.shape)
    acc = rng.normal(size=(3,) + w.n) * 5
    for axis in range(6):
        f = f0.copy()
        if axis < 3:
            speed, tau, h, per = grid.vc(axis), 0.37, grid.dx[axis], True
        else:
            speed, tau, h, per = acc[axis - 3], 0.11, grid.dv[axis - 3], False
        O.sweep(f, axis, speed, tau, h, per)
        moved = np.moveaxis(f0, axis, -1)
        got = np.moveaxis(f, axis, -1)
        for idx in np.ndindex(moved.shape[:-1]):
            full = list(idx[:axis]) + [0] + list(idx[axis:])
            if axis < 3:
                u = speed[full[3 + axis]]
            else:
                u = speed[tuple(full[:3])]
            ref = O.pfc_line(moved[idx], u * tau / h, per)
            assert np.array_equal(got[idx], ref)


def test_free_streaming_integer_courant_is_exact_shift():
    # G = 0: kicks vanish.  dt = 2 dx / dv makes v_j dt / dx = 2j + 1 - Nv.
    w = I.small_maxwell(n=(6, 5, 4), nv=(4, 6, 2), G=0.0)
    w = w.replace(vlo=(-2.0, -3.0, -1.0), vhi=(2.0, 3.0, 1.0))
    grid = O.Grid.of(w)
    rng = np.random.default_rng(1)
    f0 = rng.random(w.shape)
    dts = [2 * grid.dx[a] / grid.dv[a] for a in range(3)]
    for a in range(3):
        f = f0.copy()
        O.sweep(f, a, grid.vc(a), dts[a], grid.dx[a], True)
        expect = np.empty_like(f0)
        for j in range(w.nv[a]):
            s = 2 * j + 1 - w.nv[a]
            sl = [slice(None)] * 6
            sl[3 + a] = j
            expect[tuple(sl)] = np.roll(f0[tuple(sl)], s, axis=a)
        assert np.allclose(f, expect, rtol=0, atol=1e-14)


def test_top_hat_returns_after_one_period():
    # Test 1 (Sec. 3.1): periodic free streaming; with an integer shift per
    # step the profile is translated exactly and returns after N/|s| steps.
    f, x, v = I.top_hat_1d(32, 16)
    f6 = f.reshape(32, 1, 1, 16, 1, 1).copy()
    dv = v[1] - v[0]
    dx = x[1] - x[0]
    dt = dx / dv          # shift per step = v_j / dv = j + 1/2 - 8: half-integers
    dt = 2 * dt           # -> odd integers
    for _ in range(32):
        O.sweep(f6, 0, v, dt, dx, True)
    assert np.allclose(f6.reshape(32, 16), f, atol=1e-13)


def test_step_conserves_mass_and_positivity():
    w = I.small_maxwell(amp=0.3, G=30.0)
    sim = O.Simulation(I.initial_condition(w), O.Grid.of(w), O.Params.of(w))
    M0 = sim.energy()[0]
    sim.step(3)
    M, K, U, E, Mout = sim.energy()
    assert sim.f.min() >= 0.0
    assert abs(M + Mout - M0) <= 1e-13 * M0
    assert Mout > 0                     # the strong field pushes mass out


def test_step_without_gravity_is_the_drift():
    w = I.small_maxwell(G=0.0)
    grid = O.Grid.of(w)
    f0 = I.initial_condition(w)
    sim = O.Simulation(f0, grid, O.Params.of(w))
    dt = sim.dt()
    sim.step(1)
    f = f0.copy()
    for a in (2, 1, 0):
        O.sweep(f, a, grid.vc(a), dt, grid.dx[a], True)
    assert np.array_equal(sim.f, f)


# ---------------------------------------------------------------------------
# linear theory (Sec. 3.2, Eq. dispersion): k^2/k_J^2 = 1 + w Z(w)
# ---------------------------------------------------------------------------

def growth_root(k_over_kj):
    """Jeans growth: w = i y, w Z(w) = -sqrt(pi) y erfcx(y); gamma = y sqrt(2) k sigma."""
    return brentq(lambda y: 1 - math.sqrt(math.pi) * y * erfcx(y) - k_over_kj ** 2, 1e-9, 50)


def damping_root(k_over_kj):
    """Landau damping: w = -i y, w Z(w) = sqrt(pi) y exp(y^2) (1 + erf y)."""
    return brentq(lambda y: 1 + math.sqrt(math.pi) * y * math.exp(y * y) * (1 + erf(y))
                  - k_over_kj ** 2, 1e-12, 5)


def test_dispersion_roots_against_faddeeva():
    from scipy.special import wofz
    for kk in (0.1, 0.5):
        y = growth_root(kk)
        w = 1j * y
        Z = 1j * math.sqrt(math.pi) * wofz(w)
        assert abs(1 + w * Z - kk ** 2) < 1e-10
    for kk in (1.1, 1.5, 2.0):
        y = damping_root(kk)
        w = -1j * y
        Z = 1j * math.sqrt(math.pi) * wofz(w)
        assert abs(1 + w * Z - kk ** 2) < 1e-9


def run_1d(k_over_kj, amp, nx, nv, t_end, n_mode=2, courant=0.5):
    """Test 2 set-up (Sec. 3.2) embedded in 6D with one cell along y, z, vy,
    vz: L = 1, G = 1, rho_bar = 1 (T = 1), v in [-V, V] with V = L/T."""
    L, G, rho_bar = 1.0, 1.0, 1.0
    k = 2 * math.pi * n_mode / L
    kj = k / k_over_kj
    sigma = math.sqrt(4 * math.pi * G * rho_bar) / kj
    V = 1.0
    grid = O.Grid((nx, 1, 1), (nv, 1, 1), (-L / 2, -0.5, -0.5), (L / 2, 0.5, 0.5),
                  (-V, -0.5, -0.5), (V, 0.5, 0.5))
    x = grid.lo[0] + (np.arange(nx) + 0.5) * grid.dx[0]
    v = grid.vc(0)
    f1 = rho_bar * (1 + amp * np.cos(k * x))[:, None] * np.exp(-v ** 2 / (2 * sigma ** 2))[None, :] \
        / math.sqrt(2 * math.pi * sigma ** 2)
    f = f1.reshape(nx, 1, 1, nv, 1, 1)
    sim = O.Simulation(f, grid, O.Params(G=G, courant=courant))
    ts, amps, es = [], [], []
    while sim.t < t_end:
        rho = O.density(sim.f, grid).reshape(-1)
        ts.append(sim.t)
        amps.append(abs(np.fft.fft(rho / rho.mean() - 1)[n_mode]) * 2 / nx)
        es.append(sim.energy())
        sim.step()
    return np.array(ts), np.array(amps), es, sigma, k


@pytest.mark.slow
def test_jeans_growth_rate_matches_linear_theory():
    kk = 0.5
    ts, amps, es, sigma, k = run_1d(kk, 0.01, 64, 128, 0.9)
    gamma = growth_root(kk) * math.sqrt(2) * k * sigma
    sel = (ts > 0.3) & (ts < 0.9)
    slope = np.polyfit(ts[sel], np.log(amps[sel]), 1)[0]
    assert slope == pytest.approx(gamma, rel=0.05)


@pytest.mark.slow
def test_landau_damping_rate_matches_linear_theory():
    kk = 1.5
    # the least-damped root dominates once the initial transient (the density
    # starts with zero time derivative) has passed; the next root (about five
    # times more damped) beats with it, so fit over more than one beat
    ts, amps, es, sigma, k = run_1d(kk, 0.01, 64, 128, 0.85)
    gamma = damping_root(kk) * math.sqrt(2) * k * sigma
    sel = (ts > 0.25) & (ts < 0.8)
    slope = np.polyfit(ts[sel], np.log(amps[sel]), 1)[0]
    assert -slope == pytest.approx(gamma, rel=0.07)


@pytest.mark.slow
def test_energy_and_mass_conservation_test2():
    # Sec. 3.2: E within 1e-3 and M within 1e-6 (k/k_J = 0.5, 128 x 128),
    # checked up to t = 1.75 T; past 2 T the sheet that collapses is under-
    # resolved on 128 cells and the energy error grows past 1e-3
    T2 = golden("paper_test2")
    ts, amps, es, sigma, k = run_1d(0.5, T2["amplitude_below_kJ"], int(T2["nx"]), int(T2["nv"]),
                                    1.75)
    E0, M0 = es[0][3], es[0][0]
    dE = max(abs(e[3] - E0) for e in es) / abs(E0)
    dM = max(abs(e[0] - M0) for e in es) / M0
    assert dE < T2["energy_rel_bound"]
    assert dM < T2["mass_rel_bound"]


def test_white_noise_workloads_have_the_papers_jeans_wave_numbers():
    """The Test 4 workloads (Sec. 3.4): rho_bar, G and sigma of the synthetic
    boxes give the two Jeans wave numbers the paper prints."""
    T4 = golden("paper_test4")
    for kj_over_k1, kjl in zip((4.0, 8.0), T4["kJ_times_L_over_pi"]):
        w = I.white_noise32(kj_over_k1)
        L = w.box_hi[0] - w.box_lo[0]
        kj = math.sqrt(4 * math.pi * w.G * w.rho_bar) / w.sigma
        assert kj * L / math.pi == pytest.approx(kjl, rel=1e-12)
