"""Plain FP64 CPU oracle of the split Vlasov--Poisson step.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import this module.  It shares no code
with the CUDA path (it never imports the package's binding or kernels); the
only module both use is the seeded input generator.

What it computes, in the paper's order (Yoshikawa, Yoshida & Umemura 2013):
  * Sec. 2.1: the PFC line update and the sweeps T_l (C, vp_oracle.c);
  * Sec. 2.1, Eq. (integration): one step
        f^{n+1} = T_vz T_vy T_vx(dt/2) T_x T_y T_z(dt) T_vz T_vy T_vx(dt/2) f^n
    (operators act right to left), with the Poisson solve after the drifts;
  * Sec. 2.2: rho = integral of f over velocity; periodic Poisson by FFT with
    the discrete Green's function G(k) = -pi G Delta^2 / sum sin^2(k Delta/2);
    isolated Poisson by Hockney's doubling with G(r) = -G/r; force by the
    2-point central difference;
  * Sec. 2.4: dt = C min(dt_p, dt_v);
  * Sec. 3.1 / 3.2: diagnostics M, K, U, E.
numpy's FFT serves as the FFT step.

Readings where the paper is silent or garbled:
  * G(k = 0) = 0 (the mean density does not source the periodic potential);
  * for unequal spacings the periodic Green's function is the one of the same
    7-point Laplacian, -pi G / sum_l sin^2(k_l D_l / 2) / D_l^2;
  * the isolated kernel is -G/r (the printed +G/r has the sign garbled); at
    r = 0 it is the mean of -G/r over one cell, computed here by quadrature;
  * the isolated force stencil takes its outside neighbours from the doubled
    grid (they are exact free-space potentials);
  * V^max_l = max(|V^-_l|, |V^+_l|); dt_v uses the acceleration the first half
    kick uses, and both half kicks of a step use the same dt;
  * the state carried between steps is (f, g): g^{n+1} is computed after the
    drift of step n and serves the second half kick of step n and the first
    of step n+1;
  * K uses the cell-centre velocity.

The adjoint (not in the paper) reverses this step with the limiter branches
frozen (vp_oracle.c) and a fixed dt.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_vp.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile vp_oracle.c with gcc into liboracle_vp.so (OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            lp = ctypes.POINTER(ctypes.c_long)
            L.oracle_pfc_line.argtypes = [dp, dp, ctypes.c_long, ctypes.c_double, ctypes.c_int]
            L.oracle_pfc_line.restype = None
            L.oracle_pfc_line_adjoint.argtypes = [dp, dp, dp, ctypes.c_long, ctypes.c_double,
                                                  ctypes.c_int]
            L.oracle_pfc_line_adjoint.restype = ctypes.c_double
            L.oracle_sweep.argtypes = [dp, lp, ctypes.c_int, dp, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int]
            L.oracle_sweep.restype = ctypes.c_double
            L.oracle_sweep_adjoint.argtypes = [dp, dp, lp, ctypes.c_int, dp, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_int, dp]
            L.oracle_sweep_adjoint.restype = None
            L.oracle_pfc_line_ghosted.argtypes = [dp, dp, ctypes.c_long, ctypes.c_long,
                                                  ctypes.c_double, ctypes.c_double]
            L.oracle_pfc_line_ghosted.restype = None
            L.oracle_sweep_x_ghosted.argtypes = [dp, dp, dp, dp, lp, ctypes.c_long, dp,
                                                 ctypes.c_double, ctypes.c_double, dp]
            L.oracle_sweep_x_ghosted.restype = None
            L.oracle_density.argtypes = [dp, ctypes.c_long, ctypes.c_long, ctypes.c_double, dp]
            L.oracle_density.restype = None
            L.oracle_moments.argtypes = [dp, ctypes.c_long, ctypes.c_long, dp, dp]
            L.oracle_moments.restype = None
            L.oracle_threads.argtypes = []
            L.oracle_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def threads() -> int:
    """Threads the oracle's parallel loops run on."""
    return int(lib().oracle_threads())


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------------------
# 1D and sweep level (Sec. 2.1)
# ---------------------------------------------------------------------------

def pfc_line(f: np.ndarray, alpha: float, periodic: bool) -> np.ndarray:
    """One PFC update of a line of cell averages, shift alpha = u dt / dx."""
    a = np.ascontiguousarray(f, dtype=np.float64).copy()
    out = np.empty_like(a)
    lib().oracle_pfc_line(_dptr(a), _dptr(out), a.size, float(alpha), int(bool(periodic)))
    return out


def pfc_line_adjoint(f, lam_out, alpha, periodic):
    """(lam_in, dJ/dalpha) of pfc_line at input f for output cotangent lam_out."""
    a = np.ascontiguousarray(f, dtype=np.float64).copy()
    lo = np.ascontiguousarray(lam_out, dtype=np.float64).copy()
    li = np.empty_like(a)
    d = lib().oracle_pfc_line_adjoint(_dptr(a), _dptr(lo), _dptr(li), a.size, float(alpha),
                                      int(bool(periodic)))
    return li, d


def _dims(f: np.ndarray):
    assert f.ndim == 6
    return (ctypes.c_long * 6)(*f.shape)


def sweep(f: np.ndarray, axis: int, speed: np.ndarray, tau: float, h: float,
          periodic: bool) -> float:
    """T_axis(tau) in place on f[x][y][z][vx][vy][vz] (Sec. 2.1, Eqs.
    (adv_xpos)-(adv_zvel): the 1D update applied to every line along the
    axis).  speed: cell-centre velocities (position axis) or accelerations on
    the spatial grid (velocity axis).  Returns the phase-space sum of f that
    left through outflow faces."""
    sp = np.ascontiguousarray(speed, dtype=np.float64).reshape(-1)
    return lib().oracle_sweep(_dptr(f), _dims(f), int(axis), _dptr(sp), float(tau), float(h),
                              int(bool(periodic)))


def pfc_line_ghosted(ext: np.ndarray, n: int, G: int, alpha: float, finf: float) -> np.ndarray:
    """The update of the n cells ext[G:G+n] of a piece of a longer line whose
    G neighbouring cells on each side are ext[:G] and ext[G+n:] and whose
    maximum is finf (Sec. 2.1 on a line split across the slabs of Sec. 2.3);
    with G >= floor(|alpha|) + 2 it equals the whole-line update there."""
    e = np.ascontiguousarray(ext, dtype=np.float64)
    assert e.size == n + 2 * G
    out = np.empty(n)
    lib().oracle_pfc_line_ghosted(_dptr(e), _dptr(out), n, G, float(alpha), float(finf))
    return out


def sweep_x_ghosted(f: np.ndarray, glo: np.ndarray, ghi: np.ndarray, speed: np.ndarray,
                    tau: float, h: float, lmax: np.ndarray) -> np.ndarray:
    """T_x(tau) of a slab of x planes f[nx][ny][nz][nvx][nvy][nvz] whose x
    lines continue into the G planes glo below and ghi above it (periodic
    wrap included by whoever filled them) and have the maxima lmax
    [ny][nz][nvx][nvy][nvz] over the whole line (Sec. 2.3's decomposition of
    position space).  Returns the slab's updated planes."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    glo = np.ascontiguousarray(glo, dtype=np.float64)
    ghi = np.ascontiguousarray(ghi, dtype=np.float64)
    lm = np.ascontiguousarray(lmax, dtype=np.float64)
    G = glo.shape[0]
    assert glo.shape == ghi.shape == (G,) + f.shape[1:] and lm.shape == f.shape[1:]
    out = np.empty_like(f)
    sp = np.ascontiguousarray(speed, dtype=np.float64).reshape(-1)
    lib().oracle_sweep_x_ghosted(_dptr(f), _dptr(glo), _dptr(ghi), _dptr(out), _dims(f), G,
                                 _dptr(sp), float(tau), float(h), _dptr(lm))
    return out


def sweep_adjoint(fin: np.ndarray, lam: np.ndarray, axis: int, speed: np.ndarray, tau: float,
                  h: float, periodic: bool, dspeed: Optional[np.ndarray] = None) -> None:
    """Frozen-branch adjoint of `sweep` (not in the paper): lam (the
    cotangent of the sweep's output) is replaced by that of its input fin;
    with dspeed, the derivative with respect to each line's speed is added
    there (one entry per spatial cell for a velocity axis)."""
    sp = np.ascontiguousarray(speed, dtype=np.float64).reshape(-1)
    dp = None
    if dspeed is not None:
        assert dspeed.dtype == np.float64 and dspeed.flags.c_contiguous
        dp = _dptr(dspeed)
    lib().oracle_sweep_adjoint(_dptr(fin), _dptr(lam), _dims(fin), int(axis), _dptr(sp),
                               float(tau), float(h), int(bool(periodic)), dp)


# ---------------------------------------------------------------------------
# grid
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Grid:
    """The phase-space grid of Sec. 2: N_x N_y N_z cells on [lo, hi) and
    N^v cells per velocity axis on [V^-, V^+), values as cell averages."""
    n: Tuple[int, int, int]
    nv: Tuple[int, int, int]
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]
    vlo: Tuple[float, float, float]
    vhi: Tuple[float, float, float]

    @classmethod
    def of(cls, w) -> "Grid":
        return cls(tuple(w.n), tuple(w.nv), tuple(w.box_lo), tuple(w.box_hi), tuple(w.vlo),
                   tuple(w.vhi))

    @property
    def dx(self):
        return [(self.hi[a] - self.lo[a]) / self.n[a] for a in range(3)]

    @property
    def dv(self):
        return [(self.vhi[a] - self.vlo[a]) / self.nv[a] for a in range(3)]

    def vc(self, a):
        """Velocity cell centres along axis a (Sec. 2: V^- + (j + 1/2) dv)."""
        return self.vlo[a] + (np.arange(self.nv[a]) + 0.5) * self.dv[a]

    @property
    def dvol_x(self):
        return float(np.prod(self.dx))

    @property
    def dvol_v(self):
        return float(np.prod(self.dv))


# ---------------------------------------------------------------------------
# density, Poisson, force, timestep (Sec. 2.2, 2.4)
# ---------------------------------------------------------------------------

def density(f: np.ndarray, grid: Grid) -> np.ndarray:
    """rho(x) = sum over velocity cells of f dv_x dv_y dv_z (Sec. 2.2),
    compensated."""
    np_ = int(np.prod(grid.n))
    nv = int(np.prod(grid.nv))
    rho = np.empty(np_)
    lib().oracle_density(_dptr(f), np_, nv, grid.dvol_v, _dptr(rho))
    return rho.reshape(grid.n)


def green_periodic(grid: Grid, G: float) -> np.ndarray:
    """Green's function of the periodic solve in k space (Sec. 2.2): the
    discrete one of the 7-point Laplacian, -pi G / sum_l sin^2(k_l dx_l / 2)
    / dx_l^2, and 0 at k = 0."""
    s = np.zeros(grid.n)
    for a in range(3):
        m = np.fft.fftfreq(grid.n[a]) * grid.n[a]          # integer wave numbers
        k = 2 * np.pi * m / (grid.n[a] * grid.dx[a])
        sh = [1, 1, 1]
        sh[a] = grid.n[a]
        s = s + (np.sin(k * grid.dx[a] / 2) ** 2 / grid.dx[a] ** 2).reshape(sh)
    with np.errstate(divide="ignore", invalid="ignore"):
        g = -np.pi * G / s
    g[0, 0, 0] = 0.0
    return g


def cube_mean_inverse_distance() -> float:
    """Mean of 1/r over the unit cube centred on r = 0, by quadrature: the
    integral over z is done in closed form (asinh), the rest with scipy."""
    from scipy.integrate import dblquad
    val, _ = dblquad(lambda y, x: math.asinh(0.5 / math.hypot(x, y)) if (x or y) else 0.0,
                     0.0, 0.5, 0.0, 0.5, epsabs=1e-13, epsrel=1e-13)
    return 8.0 * val


def green_isolated(grid: Grid, G: float) -> np.ndarray:
    """Hockney's doubled kernel in real space (Sec. 2.2): -G/r on 0..N per
    axis, mirrored onto N+1..2N-1.  Needs equal spacings for the r = 0 cell."""
    dx = grid.dx
    if not (abs(dx[0] - dx[1]) < 1e-12 * dx[0] and abs(dx[0] - dx[2]) < 1e-12 * dx[0]):
        raise ValueError("isolated Poisson needs cubic cells")
    axes = []
    for a in range(3):
        i = np.arange(2 * grid.n[a])
        axes.append(np.minimum(i, 2 * grid.n[a] - i) * dx[a])
    r = np.sqrt(axes[0][:, None, None] ** 2 + axes[1][None, :, None] ** 2
                + axes[2][None, None, :] ** 2)
    with np.errstate(divide="ignore"):
        g = -G / r
    g[0, 0, 0] = -G * cube_mean_inverse_distance() / dx[0]
    return g


def poisson(rho: np.ndarray, grid: Grid, G: float, bc: str,
            ghat: Optional[np.ndarray] = None) -> np.ndarray:
    """phi from rho by FFT convolution (Sec. 2.2).  Periodic: phi =
    IFFT(G(k) FFT(rho)).  Isolated: Hockney's doubled-grid convolution with
    the -G/r kernel; returns phi on the whole 2N grid."""
    if bc == "periodic":
        gk = green_periodic(grid, G) if ghat is None else ghat
        return np.real(np.fft.ifftn(gk * np.fft.fftn(rho)))
    n = grid.n
    big = np.zeros(tuple(2 * m for m in n))
    big[:n[0], :n[1], :n[2]] = rho
    gk = np.fft.fftn(green_isolated(grid, G)) if ghat is None else ghat
    return np.real(np.fft.ifftn(gk * np.fft.fftn(big))) * grid.dvol_x


def force(phi: np.ndarray, grid: Grid, bc: str) -> np.ndarray:
    """g = -grad phi by the 2-point central difference (Sec. 2.2).  Returns
    shape (3, Nx, Ny, Nz)."""
    g = np.empty((3,) + tuple(grid.n))
    for a in range(3):
        if bc == "periodic":
            d = np.roll(phi, -1, axis=a) - np.roll(phi, 1, axis=a)
        else:   # isolated: phi lives on the doubled grid; index -1 is 2N-1
            d = np.roll(phi, -1, axis=a) - np.roll(phi, 1, axis=a)
            d = d[:grid.n[0], :grid.n[1], :grid.n[2]]
        g[a] = -d / (2 * grid.dx[a])
    return g


def potential_in_box(phi: np.ndarray, grid: Grid) -> np.ndarray:
    """The part of phi on the physical box (the whole array when periodic)."""
    return phi[:grid.n[0], :grid.n[1], :grid.n[2]]


def timestep(g: np.ndarray, grid: Grid, courant: float) -> float:
    """dt = C min(dt_p, dt_v) (Sec. 2.4)."""
    dtp = min(grid.dx[a] / max(abs(grid.vlo[a]), abs(grid.vhi[a])) for a in range(3))
    dtv = math.inf
    for a in range(3):
        amax = float(np.max(np.abs(g[a])))
        if amax > 0:
            dtv = min(dtv, grid.dv[a] / amax)
    return courant * min(dtp, dtv)


# ---------------------------------------------------------------------------
# the split step (Sec. 2.1, Eq. integration)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    """G, the Courant number C (Sec. 2.4), a fixed dt (> 0) or adaptive, and
    the boundary rules of Sec. 2.1 (position sweeps) and Sec. 2.2 (Poisson)."""
    G: float = 1.0
    courant: float = 0.5
    dt_fixed: float = 0.0
    space_bc: str = "periodic"
    poisson_bc: str = "periodic"

    @classmethod
    def of(cls, w) -> "Params":
        return cls(w.G, w.courant, w.dt_fixed, w.space_bc, w.poisson_bc)


class Simulation:
    """f (FP64) with its acceleration g; `step` is one split step of
    Eq. (integration), read right to left: half kick vx, vy, vz with g^n,
    drift z, y, x, field of the drifted f, half kick with g^{n+1}."""

    def __init__(self, f: np.ndarray, grid: Grid, params: Params, copy: bool = True):
        """copy=False adopts f itself when it is a contiguous FP64 array (a
        69 GB state would otherwise be held twice); the steps then update it
        in place."""
        self.grid = grid
        self.p = params
        c = np.ascontiguousarray(f, dtype=np.float64)
        self.f = c.copy() if (copy and c is f) else c
        self.t = 0.0
        self.lost = 0.0                  # phase-space sum that left (unscaled)
        self.ghat = None
        if params.poisson_bc == "isolated":
            self.ghat = np.fft.fftn(green_isolated(grid, params.G))
        self.rho, self.phi, self.g = self.field(self.f)

    def field(self, f):
        """rho, phi and g = -grad phi of f (Sec. 2.2)."""
        rho = density(f, self.grid)
        phi = poisson(rho, self.grid, self.p.G, self.p.poisson_bc, self.ghat)
        g = force(phi, self.grid, self.p.poisson_bc)
        return rho, phi, g

    def dt(self) -> float:
        """The fixed dt, or C min(dt_p, dt_v) from the current g (Sec. 2.4)."""
        if self.p.dt_fixed > 0:
            return self.p.dt_fixed
        return timestep(self.g, self.grid, self.p.courant)

    def kick(self, g, tau):
        """T_vz T_vy T_vx(tau) with acceleration g (Sec. 2.1, outflow in v)."""
        for a in range(3):                                   # vx, vy, vz
            self.lost += sweep(self.f, 3 + a, g[a], tau, self.grid.dv[a], False)

    def drift(self, tau):
        """T_x T_y T_z(tau) with the cell-centre velocities (Sec. 2.1)."""
        per = self.p.space_bc == "periodic"
        for a in (2, 1, 0):                                  # z, y, x
            self.lost += sweep(self.f, a, self.grid.vc(a), tau, self.grid.dx[a], per)

    def step(self, n: int = 1):
        for _ in range(n):
            dt = self.dt()
            self.kick(self.g, dt / 2)
            self.drift(dt)
            self.rho, self.phi, self.g = self.field(self.f)
            self.kick(self.g, dt / 2)
            self.t += dt
        return self.t

    def energy(self):
        """(M, K, U, E, M_out): Sec. 3.1 Eqs. (kinetic_energy), (total_mass),
        Sec. 3.2 U = 1/2 int rho phi; M_out is the mass that left."""
        return energy(self.f, self.grid, self.p, self.ghat) + (self.lost * self.grid.dvol_x
                                                                * self.grid.dvol_v,)


def velocity_square(grid: Grid) -> np.ndarray:
    """|v|^2 at the velocity cell centres (the K of Sec. 3.1)."""
    vx, vy, vz = (grid.vc(a) for a in range(3))
    return (vx[:, None, None] ** 2 + vy[None, :, None] ** 2 + vz[None, None, :] ** 2).reshape(-1)


def energy(f: np.ndarray, grid: Grid, p: Params, ghat=None):
    """(M, K, U, E) of f: Sec. 3.1 Eqs. (total_mass), (kinetic_energy) with
    cell-centre velocities, Sec. 3.2 U = 1/2 sum rho phi dV_x, E = K + U."""
    np_ = int(np.prod(grid.n))
    nv = int(np.prod(grid.nv))
    v2 = velocity_square(grid)
    out = np.empty(2)
    lib().oracle_moments(_dptr(f), np_, nv, _dptr(v2), _dptr(out))
    M = out[0] * grid.dvol_x * grid.dvol_v
    K = 0.5 * out[1] * grid.dvol_x * grid.dvol_v
    rho = density(f, grid)
    phi = poisson(rho, grid, p.G, p.poisson_bc, ghat)
    U = 0.5 * float(np.sum(rho * potential_in_box(phi, grid))) * grid.dvol_x
    return M, K, U, K + U


# ---------------------------------------------------------------------------
# adjoint (not in the paper): reverse of Simulation.step with fixed dt
# ---------------------------------------------------------------------------

def poisson_adjoint(lam_phi: np.ndarray, grid: Grid, G: float, bc: str, ghat=None):
    """Transpose of `poisson` (its kernel is symmetric).  For the isolated case
    lam_phi lives on the doubled grid and the result on the box."""
    if bc == "periodic":
        gk = green_periodic(grid, G) if ghat is None else ghat
        return np.real(np.fft.ifftn(np.conj(gk) * np.fft.fftn(lam_phi)))
    gk = np.fft.fftn(green_isolated(grid, G)) if ghat is None else ghat
    full = np.real(np.fft.ifftn(np.conj(gk) * np.fft.fftn(lam_phi))) * grid.dvol_x
    return full[:grid.n[0], :grid.n[1], :grid.n[2]]


def force_adjoint(lam_g: np.ndarray, grid: Grid, bc: str, shape_phi) -> np.ndarray:
    """Transpose of `force`: lam_phi from lam_g (3, N...)."""
    lam_phi = np.zeros(shape_phi)
    for a in range(3):
        c = -lam_g[a] / (2 * grid.dx[a])
        if bc == "periodic":
            lam_phi += np.roll(c, 1, axis=a) - np.roll(c, -1, axis=a)
        else:
            big = np.zeros(shape_phi)
            big[:grid.n[0], :grid.n[1], :grid.n[2]] = c
            lam_phi += np.roll(big, 1, axis=a) - np.roll(big, -1, axis=a)
    return lam_phi


def density_adjoint(lam_rho: np.ndarray, grid: Grid) -> np.ndarray:
    """Transpose of `density`: broadcast lam_rho dvol_v over velocity."""
    nv = int(np.prod(grid.nv))
    out = np.repeat(lam_rho.reshape(-1, 1) * grid.dvol_v, nv, axis=1)
    return out.reshape(tuple(grid.n) + tuple(grid.nv))


def field_adjoint(lam_g: np.ndarray, sim: "Simulation") -> np.ndarray:
    """lam_f contribution of g = force(poisson(density(f)))."""
    grid, p = sim.grid, sim.p
    shape_phi = grid.n if p.poisson_bc == "periodic" else tuple(2 * m for m in grid.n)
    lam_phi = force_adjoint(lam_g, grid, p.poisson_bc, shape_phi)
    lam_rho = poisson_adjoint(lam_phi, grid, p.G, p.poisson_bc, sim.ghat)
    return density_adjoint(lam_rho, grid)


def adjoint_step(sim: "Simulation", f_n: np.ndarray, g_n: np.ndarray,
                 lam_f: np.ndarray, lam_g: np.ndarray):
    """Given the step-start state (f_n, g_n) and the cotangents of the
    step-end state (f^{n+1}, g^{n+1}), return those of (f_n, g_n).  Uses
    sim.p.dt_fixed (required > 0)."""
    grid, p = sim.grid, sim.p
    if p.dt_fixed <= 0:
        raise ValueError("the adjoint needs a fixed dt")
    dt = p.dt_fixed
    per = p.space_bc == "periodic"
    # forward replay, keeping every sweep input
    f = np.ascontiguousarray(f_n, dtype=np.float64).copy()
    inputs: List[Tuple[np.ndarray, int, np.ndarray, float, float, bool, str]] = []

    def fwd(axis, speed, tau, h, periodic, tag):
        inputs.append((f.copy(), axis, speed, tau, h, periodic, tag))
        sweep(f, axis, speed, tau, h, periodic)

    for a in range(3):
        fwd(3 + a, g_n[a], dt / 2, grid.dv[a], False, "k1")
    for a in (2, 1, 0):
        fwd(a, grid.vc(a), dt, grid.dx[a], per, "d")
    f_b = f.copy()
    _, _, g_new = sim.field(f_b)
    for a in range(3):
        fwd(3 + a, g_new[a], dt / 2, grid.dv[a], False, "k2")
    lam = np.ascontiguousarray(lam_f, dtype=np.float64).copy()
    lam_g_new = np.ascontiguousarray(lam_g, dtype=np.float64).copy()
    lam_g_n = np.zeros_like(lam_g_new)
    for fin, axis, speed, tau, h, periodic, tag in reversed(inputs):
        if tag == "k2":
            ds = np.zeros(int(np.prod(grid.n)))
            sweep_adjoint(fin, lam, axis, speed, tau, h, periodic, ds)
            lam_g_new[axis - 3] += ds.reshape(grid.n)
            if axis == 3:          # all of K2 reversed: g^{n+1} came from f_b
                lam += field_adjoint(lam_g_new, sim)
        elif tag == "k1":
            ds = np.zeros(int(np.prod(grid.n)))
            sweep_adjoint(fin, lam, axis, speed, tau, h, periodic, ds)
            lam_g_n[axis - 3] += ds.reshape(grid.n)
        else:
            sweep_adjoint(fin, lam, axis, speed, tau, h, periodic, None)
    return lam, lam_g_n


def field_energy_gradient(f: np.ndarray, sim: "Simulation") -> Tuple[float, np.ndarray]:
    """J = U = 1/2 sum rho phi dV_x and dJ/df (phi dV_x broadcast with dV_v)."""
    grid, p = sim.grid, sim.p
    rho = density(f, grid)
    phi = poisson(rho, grid, p.G, p.poisson_bc, sim.ghat)
    phib = potential_in_box(phi, grid)
    J = 0.5 * float(np.sum(rho * phib)) * grid.dvol_x
    return J, density_adjoint(phib * grid.dvol_x, grid)


def density_misfit_gradient(f: np.ndarray, sim: "Simulation", target: np.ndarray):
    """J = 1/2 sum (rho - target)^2 dV_x and dJ/df."""
    grid = sim.grid
    rho = density(f, grid)
    r = rho - target
    J = 0.5 * float(np.sum(r * r)) * grid.dvol_x
    return J, density_adjoint(r * grid.dvol_x, grid)
