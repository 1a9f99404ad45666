"""Pins of the oracle's density, Poisson, force and timestep (Sec. 2.2, 2.4)
against closed forms, the discrete Laplacian and brute-force sums."""
import math

import numpy as np
import pytest

from oracle import vp_oracle as O


def _grid(n, box, nv=(3, 2, 2)):
    return O.Grid(tuple(n), tuple(nv), tuple(-b / 2 for b in box), tuple(b / 2 for b in box),
                  (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))


def laplacian7(phi, dx):
    out = np.zeros_like(phi)
    for a in range(3):
        out += (np.roll(phi, -1, a) - 2 * phi + np.roll(phi, 1, a)) / dx[a] ** 2
    return out


@pytest.mark.parametrize("n,box", [((8, 8, 8), (1, 1, 1)), ((6, 10, 5), (1.0, 1.3, 0.7))])
def test_periodic_poisson_solves_7point_laplacian(n, box):
    g = _grid(n, box)
    rng = np.random.default_rng(0)
    rho = rng.random(n)
    G = 1.7
    phi = O.poisson(rho, g, G, "periodic")
    lap = laplacian7(phi, g.dx)
    assert np.allclose(lap, 4 * math.pi * G * (rho - rho.mean()), rtol=0, atol=1e-11 * rho.max())
    assert abs(phi.mean()) < 1e-13


def test_periodic_poisson_single_mode_closed_form():
    n, L = 16, 2.0
    g = _grid((n, 4, 4), (L, 0.5, 0.5))
    x = g.lo[0] + (np.arange(n) + 0.5) * g.dx[0]
    k = 2 * math.pi * 3 / L
    rho = np.broadcast_to(np.cos(k * x)[:, None, None], g.n).copy()
    phi = O.poisson(rho, g, 1.0, "periodic")
    keff2 = (2 / g.dx[0] * math.sin(k * g.dx[0] / 2)) ** 2
    assert np.allclose(phi, -4 * math.pi * rho / keff2, atol=1e-13)


def test_cube_mean_inverse_distance_closed_form():
    # mean of 1/r over the unit cube about its centre: 3 ln(2 + sqrt 3) - pi/2
    assert O.cube_mean_inverse_distance() == pytest.approx(
        3 * math.log(2 + math.sqrt(3)) - math.pi / 2, rel=1e-10)


def test_isolated_poisson_matches_direct_sum():
    n = (5, 4, 6)
    d = 0.3
    g = O.Grid(n, (2, 2, 2), tuple(-m * d / 2 for m in n), tuple(m * d / 2 for m in n),
               (-1,) * 3, (1,) * 3)
    rng = np.random.default_rng(1)
    rho = rng.random(n)
    G = 0.9
    phi_big = O.poisson(rho, g, G, "isolated")
    idx = np.array(np.meshgrid(*[np.arange(m) for m in n], indexing="ij")).reshape(3, -1).T
    self_term = -G * (3 * math.log(2 + math.sqrt(3)) - math.pi / 2) / d
    dvol = d ** 3

    def direct(p):
        r = np.sqrt((((idx - np.asarray(p)) * d) ** 2).sum(1))
        kern = np.where(r > 0, -G / np.where(r > 0, r, 1), self_term)
        return dvol * float(np.sum(kern * rho.reshape(-1)))

    for p in [(0, 0, 0), (4, 3, 5), (2, 1, 3), (1, 2, 0)]:
        assert phi_big[p] == pytest.approx(direct(p), rel=1e-12)
    # one layer outside the box on either side is still exact free space
    assert phi_big[n[0], 1, 2] == pytest.approx(direct((n[0], 1, 2)), rel=1e-12)
    assert phi_big[2 * n[0] - 1, 1, 2] == pytest.approx(direct((-1, 1, 2)), rel=1e-12)
    assert phi_big[3, 2 * n[1] - 1, 0] == pytest.approx(direct((3, -1, 0)), rel=1e-12)


def test_force_central_difference_closed_form():
    n, L = 12, 1.0
    g = _grid((n, n, n), (L, L, L))
    x = g.lo[0] + (np.arange(n) + 0.5) * g.dx[0]
    y = g.lo[1] + (np.arange(n) + 0.5) * g.dx[1]
    k = 2 * math.pi * 2 / L
    phi = (np.sin(k * x)[:, None, None] + np.cos(k * y)[None, :, None]) * np.ones(g.n)
    acc = O.force(phi, g, "periodic")
    h = g.dx[0]
    assert np.allclose(acc[0], -(math.sin(k * h) / h) * np.cos(k * x)[:, None, None], atol=1e-12)
    assert np.allclose(acc[1], (math.sin(k * h) / h) * np.sin(k * y)[None, :, None], atol=1e-12)
    assert np.allclose(acc[2], 0.0, atol=1e-12)


def test_timestep_closed_form():
    g = O.Grid((8, 4, 2), (4, 4, 4), (0, 0, 0), (1, 2, 3), (-2, -1, -3), (3, 1, 2))
    acc = np.zeros((3,) + g.n)
    # dt_p = min(dx / Vmax) = min(0.125/3, 0.5/1, 1.5/3)
    assert O.timestep(acc, g, 0.5) == pytest.approx(0.5 * 0.125 / 3)
    acc[1, 3, 2, 1] = -40.0       # dv_y = 0.5 -> dt_v = 0.5 / 40
    assert O.timestep(acc, g, 0.5) == pytest.approx(0.5 * 0.5 / 40)


def test_density_sums_velocity_cells():
    g = O.Grid((3, 2, 2), (4, 3, 5), (0,) * 3, (1,) * 3, (0, 0, 0), (2, 3, 1))
    rng = np.random.default_rng(2)
    f = rng.integers(0, 1000, size=g.n + g.nv).astype(np.float64)
    rho = O.density(f, g)
    dv = g.dvol_v
    assert np.array_equal(rho, f.reshape(12, -1).sum(1).reshape(g.n) * dv)


def test_kinetic_energy_and_mass_closed_form():
    """M and K (Sec. 3.1: M = sum f dV, K = 1/2 sum f |v|^2 dV with the
    cell-centre velocity) of a hand-built f, worked out by hand.

    Grid: 2 x 1 x 1 unit cells (dV_x = 1); velocity cells vx in [-3, 3) (3
    cells: centres -2, 0, 2), vy in [-1, 3) (2 cells: centres 0, 2), vz in
    [1, 2) (1 cell: centre 1.5), so dV_v = 2 * 2 * 1 = 4.  f = (x + 1)(i + 1)
    with x the position index and i the vx index, the same for both vy.
    Per x weight (x + 1): 1 + 2 = 3.  Sum over velocities of
    (i + 1)|v|^2: i = 0 (vx^2 = 4): (4 + 0 + 2.25) + (4 + 4 + 2.25) = 16.5;
    i = 1 (vx = 0): 2 * (2.25 + 6.25) = 17; i = 2: 3 * 16.5 = 49.5; total
    83.  K = 1/2 * 4 * 3 * 83 = 498.  M = 4 * 3 * (1 + 2 + 3) * 2 = 144."""
    grid = O.Grid((2, 1, 1), (3, 2, 1), (0.0, 0.0, 0.0), (2.0, 1.0, 1.0), (-3.0, -1.0, 1.0),
                  (3.0, 3.0, 2.0))
    f = np.zeros((2, 1, 1, 3, 2, 1))
    for x in range(2):
        for i in range(3):
            f[x, 0, 0, i, :, 0] = (x + 1) * (i + 1)
    M, K, U, E = O.energy(f, grid, O.Params(G=0.0))
    assert M == 144.0
    assert K == 498.0
    assert U == 0.0 and E == K
