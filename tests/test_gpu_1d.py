"""The one-dimensional tests of Sec. 3.1-3.3 (Tests 1-3) run through the 6D
GPU library on degenerate grids (one cell along y, z, vy, vz), FP64 storage:

* Test 1: periodic free streaming of a top hat (G = 0), against the oracle
  step by step, with mass, positivity and the maximum principle;
* Test 2: the linear Jeans growth rate (k/k_J = 0.5) and the gravitational
  Landau damping rate (k/k_J = 1.5) against the roots of the Maxwellian
  dispersion relation, and the density-mode amplitude against the oracle;
* Test 3: the same growth with the Maxwellian moving at v_t = sigma and
  2 sigma (Galilean invariance: the rate does not change).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = pytest.mark.skip(reason="needs a CUDA GPU")

from conftest import golden  # noqa: E402
from oracle import vp_oracle as O  # noqa: E402
from paper_1206_6152_gb300 import inputs as I  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1206_6152_gb300 import build as B
    B.build()


def sim_1d(f2, L, V, G, courant=0.5, dt_fixed=0.0):
    from paper_1206_6152_gb300.vlasov import VlasovPoisson, make_config
    nx, nv = f2.shape
    cfg = make_config((nx, 1, 1), (nv, 1, 1), (-L / 2, -0.5, -0.5), (L / 2, 0.5, 0.5),
                      (-V, -0.5, -0.5), (V, 0.5, 0.5), G=G, courant=courant, dt_fixed=dt_fixed,
                      dtype=torch.float64)
    f = torch.from_numpy(np.ascontiguousarray(f2.reshape(nx, 1, 1, nv, 1, 1))).to(DEV)
    return VlasovPoisson(cfg, f), f


def grid_1d(nx, nv, L, V):
    return O.Grid((nx, 1, 1), (nv, 1, 1), (-L / 2, -0.5, -0.5), (L / 2, 0.5, 0.5),
                  (-V, -0.5, -0.5), (V, 0.5, 0.5))


@pytest.mark.gpu
def test_top_hat_free_streaming_matches_oracle():
    nx, nv = 128, 128
    f0, x, v = I.top_hat_1d(nx, nv)
    dt = 0.37 * (1.0 / nx) / 1.0                    # non-integer Courant numbers
    sim, f = sim_1d(f0, 1.0, 1.0, G=0.0, dt_fixed=dt)
    ref = O.Simulation(f0.reshape(nx, 1, 1, nv, 1, 1).copy(), grid_1d(nx, nv, 1.0, 1.0),
                       O.Params(G=0.0, courant=0.5, dt_fixed=dt))
    M0 = f0.sum()
    for _ in range(5):
        sim.step(8)
        ref.step(8)
        got = f.cpu().numpy().reshape(nx, nv)
        assert np.abs(got - ref.f.reshape(nx, nv)).max() <= 1e-12
    assert abs(got.sum() - M0) <= 1e-12 * M0
    assert got.min() >= 0.0 and got.max() <= 1.0 + 1e-13
    sim.close()


def maxwell_1d(nx, nv, k_over_kj, amp, vt=0.0, n_mode=2):
    """Test 2 set-up: L = 1, G = 1, rho_bar = 1, v in [-1, 1]; sigma from k_J."""
    L, G, rho_bar, V = 1.0, 1.0, 1.0, 1.0
    k = 2 * math.pi * n_mode / L
    kj = k / k_over_kj
    sigma = math.sqrt(4 * math.pi * G * rho_bar) / kj
    x = -L / 2 + (np.arange(nx) + 0.5) * (L / nx)
    v = -V + (np.arange(nv) + 0.5) * (2 * V / nv)
    f = rho_bar * (1 + amp * np.cos(k * x))[:, None] \
        * np.exp(-(v - vt) ** 2 / (2 * sigma ** 2))[None, :] / math.sqrt(2 * math.pi * sigma ** 2)
    return f, sigma, k


def mode_amplitude(rho, n_mode=2):
    rho = np.asarray(rho).reshape(-1)
    return abs(np.fft.fft(rho / rho.mean() - 1)[n_mode]) * 2 / rho.size


def run_gpu(f0, t_end):
    sim, f = sim_1d(f0, 1.0, 1.0, G=1.0)
    ts, amps = [], []
    t = 0.0
    while t < t_end:
        ts.append(t)
        amps.append(mode_amplitude(sim.density().cpu().numpy()))
        t = sim.step(1, sync=True)
    sim.close()
    return np.array(ts), np.array(amps)


def growth_root(kk):
    from scipy.optimize import brentq
    from scipy.special import erfcx
    return brentq(lambda y: 1 - math.sqrt(math.pi) * y * erfcx(y) - kk ** 2, 1e-9, 50)


def damping_root(kk):
    from scipy.optimize import brentq
    return brentq(lambda y: 1 + math.sqrt(math.pi) * y * math.exp(y * y) * (1 + math.erf(y))
                  - kk ** 2, 1e-12, 5)


@pytest.mark.gpu
def test_jeans_growth_matches_theory_and_oracle():
    f0, sigma, k = maxwell_1d(64, 128, 0.5, 0.01)
    ts, amps = run_gpu(f0, 0.9)
    gamma = growth_root(0.5) * math.sqrt(2) * k * sigma
    sel = (ts > 0.3) & (ts < 0.9)
    assert np.polyfit(ts[sel], np.log(amps[sel]), 1)[0] == pytest.approx(gamma, rel=0.05)
    # the oracle's trajectory, first 40 steps
    ref = O.Simulation(f0.reshape(64, 1, 1, 128, 1, 1).copy(), grid_1d(64, 128, 1.0, 1.0),
                       O.Params(G=1.0, courant=0.5))
    for n in range(40):
        assert abs(ref.t - ts[n]) <= 1e-12 * max(ts[n], 1.0)
        assert mode_amplitude(O.density(ref.f, ref.grid)) == pytest.approx(amps[n], rel=1e-9)
        ref.step()


@pytest.mark.gpu
def test_landau_damping_matches_theory():
    f0, sigma, k = maxwell_1d(64, 128, 1.5, 0.01)
    ts, amps = run_gpu(f0, 0.85)
    gamma = damping_root(1.5) * math.sqrt(2) * k * sigma
    sel = (ts > 0.25) & (ts < 0.8)
    assert -np.polyfit(ts[sel], np.log(amps[sel]), 1)[0] == pytest.approx(gamma, rel=0.07)


@pytest.mark.gpu
@pytest.mark.parametrize("vt_over_sigma", [1.0, 2.0])
def test_galilean_shift_keeps_the_growth_rate(vt_over_sigma):
    f0, sigma, k = maxwell_1d(64, 128, 0.5, 0.01)
    f1, _s, _k = maxwell_1d(64, 128, 0.5, 0.01, vt=vt_over_sigma * sigma)
    t0, a0 = run_gpu(f0, 0.9)
    t1, a1 = run_gpu(f1, 0.9)
    s0 = (t0 > 0.3) & (t0 < 0.9)
    s1 = (t1 > 0.3) & (t1 < 0.9)
    g0 = np.polyfit(t0[s0], np.log(a0[s0]), 1)[0]
    g1 = np.polyfit(t1[s1], np.log(a1[s1]), 1)[0]
    assert g1 == pytest.approx(g0, rel=0.05)


# Sec. 3.2, Test 2 as the paper runs it: 128 x 128 cells, n = 2, k/k_J in
# {0.1, 0.5, 1.1, 2.0}, A = 0.01 below k_J and 0.1 above.  The density starts
# with zero time derivative, so the early slope of log |A_2| mixes the
# growing (damped) root with the others; each rate is fitted where the least
# stable root dominates (windows and tolerances chosen on the FP64 oracle:
# 3.454, 2.425, -0.580, -7.0 against 3.492, 2.436, -0.578, -6.64).  At
# k/k_J = 2.0 the velocity bound V = L/T cuts the Maxwellian at 1.8 sigma,
# hence the wider tolerance.
T2 = golden("paper_test2")
T3 = golden("paper_test3")
FIT = {0.1: ((0.5, 1.0), 0.03), 0.5: ((0.3, 1.0), 0.03), 1.1: ((0.3, 1.0), 0.03),
       2.0: ((0.1, 0.4), 0.10)}
PAPER_RUNS = [(kk, T2["amplitude_below_kJ"] if kk < 1 else T2["amplitude_above_kJ"]) + FIT[kk]
              for kk in T2["k_over_kJ"]]


@pytest.mark.gpu
@pytest.mark.parametrize("kk, amp, window, tol", PAPER_RUNS)
def test_test2_runs_of_the_paper(kk, amp, window, tol):
    nx, nv = int(T2["nx"]), int(T2["nv"])
    f0, sigma, k = maxwell_1d(nx, nv, kk, amp, n_mode=int(T2["n_mode"]))
    ts, amps = run_gpu(f0, window[1] + 0.01)
    y = growth_root(kk) if kk < 1 else -damping_root(kk)
    theory = y * math.sqrt(2) * k * sigma
    sel = (ts > window[0]) & (ts < window[1])
    slope = np.polyfit(ts[sel], np.log(amps[sel]), 1)[0]
    assert slope == pytest.approx(theory, rel=tol)
    # the same run in the oracle, first 30 steps
    ref = O.Simulation(f0.reshape(nx, 1, 1, nv, 1, 1).copy(), grid_1d(nx, nv, 1.0, 1.0),
                       O.Params(G=1.0, courant=0.5))
    for n in range(30):
        assert abs(ref.t - ts[n]) <= 1e-12 * max(ts[n], 1.0)
        assert mode_amplitude(O.density(ref.f, ref.grid)) == pytest.approx(amps[n], rel=1e-9)
        ref.step()


@pytest.mark.gpu
def test_test2_energy_and_mass_conservation():
    """Sec. 3.2: E within 1e-3 and M within 1e-6 (k/k_J = 0.5, 128 x 128), up
    to t = 1.75 T (past 2 T the collapsing sheet is under-resolved on 128
    cells and the energy error grows past 1e-3, as in the oracle)."""
    f0, sigma, k = maxwell_1d(int(T2["nx"]), int(T2["nv"]), 0.5, T2["amplitude_below_kJ"])
    sim, f = sim_1d(f0, 1.0, 1.0, G=1.0)
    e0 = sim.energy()
    dE = dM = 0.0
    t = 0.0
    while t < 1.75:
        t = sim.step(1, sync=True)
        e = sim.energy()
        dE = max(dE, abs(e["E"] - e0["E"]) / abs(e0["E"]))
        dM = max(dM, abs(e["M"] + e["M_out"] - e0["M"]) / e0["M"])
    sim.close()
    assert dE < T2["energy_rel_bound"]
    assert dM < T2["mass_rel_bound"]


@pytest.mark.gpu
def test_test3_galilean_shift_at_landau_damping():
    """Sec. 3.3 at k/k_J = 1.1 (A = 0.1): v_t = sigma keeps the damping rate.
    (At v_t = 2 sigma the bound V = L/T cuts the shifted Maxwellian at 1.2
    sigma and the outflow changes the rate by a third in the oracle as well;
    that case is not a test of the scheme.)"""
    kk, nx, nv = T3["k_over_kJ"][1], int(T3["nx"]), int(T3["nv"])
    amp = T2["amplitude_above_kJ"]
    f0, sigma, k = maxwell_1d(nx, nv, kk, amp)
    f1, _s, _k = maxwell_1d(nx, nv, kk, amp, vt=T3["vt_over_sigma"][0] * sigma)
    t0, a0 = run_gpu(f0, 1.01)
    t1, a1 = run_gpu(f1, 1.01)
    s0 = (t0 > 0.3) & (t0 < 1.0)
    s1 = (t1 > 0.3) & (t1 < 1.0)
    g0 = np.polyfit(t0[s0], np.log(a0[s0]), 1)[0]
    g1 = np.polyfit(t1[s1], np.log(a1[s1]), 1)[0]
    assert g1 == pytest.approx(g0, rel=0.03)
