"""Seeded synthetic inputs shaped like the paper's tests.

This module is shared by the CUDA path, the oracle and the tests.  It only
builds inputs: grids, initial distribution functions and their seeded
parameters.  It holds none of the integrator's arithmetic (no sweep, no
Poisson solve, no force) and imports nothing from the CUDA binding or from
the oracle.

Initial conditions (Yoshikawa, Yoshida & Umemura, Sec. 3):
  * Maxwellian with density modes (Test 2 / Test 4 form, Sec. 3.2 and 3.4):
        f = rho_bar (1 + delta(x)) (2 pi sigma^2)^{-3/2} exp(-|v|^2 / 2 sigma^2)
    with delta(x) = sum_m A_m cos(k_m . x + theta_m), sampled at cell centres.
  * King sphere (Test 5, Sec. 3.5): f(E) proportional to exp(E/sigma^2) - 1
    for E = Psi(r) - v^2/2 > 0, Psi from the lowered-isothermal (King) ODE,
    sampled at cell centres.  The virial renormalisation of Sec. 3.5 needs the
    integrator's own energies and is done by the caller.
  * Top hat in 1D+1V (Test 1, Sec. 3.1).

Workloads mirror the five configurations used for the measurements (the grid
sizes, boxes and step counts of the paper's Tests 2, 4 and 5 at GB300 scale).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np

Vec3 = Tuple[float, float, float]


@dataclasses.dataclass(frozen=True)
class Workload:
    """A phase-space grid plus the run parameters (Sec. 2, grid definition)."""

    name: str
    n: Tuple[int, int, int]            # N_x, N_y, N_z
    nv: Tuple[int, int, int]           # N^v_x, N^v_y, N^v_z
    box_lo: Vec3
    box_hi: Vec3
    vlo: Vec3
    vhi: Vec3
    G: float = 1.0
    courant: float = 0.5
    dt_fixed: float = 0.0              # > 0: fixed step; <= 0: adaptive
    space_bc: str = "periodic"         # "periodic" | "outflow"
    poisson_bc: str = "periodic"       # "periodic" | "isolated"
    dtype: str = "f32"                 # storage of f: "f32" | "f64"
    steps: int = 1
    seed: int = 0
    # initial condition
    ic: str = "maxwell"                # "maxwell" | "king" | "king2" | "noise"
    rho_bar: float = 1.0
    sigma: float = 1.0
    modes: Tuple[Tuple[Tuple[int, int, int], float, float], ...] = ()
    king_w0: float = 6.0
    noise_amp: float = 0.0             # ic "noise": rms of the white-noise density contrast
    king_sep: float = 0.0              # ic "king2": centre separation along x (r0 units)
    king_u: float = 0.0                # ic "king2": each sphere's speed towards the other

    # -- geometry (problem definition, Sec. 2) --------------------------
    @property
    def dx(self) -> Vec3:
        return tuple((h - l) / n for l, h, n in zip(self.box_lo, self.box_hi, self.n))

    @property
    def dv(self) -> Vec3:
        return tuple((h - l) / n for l, h, n in zip(self.vlo, self.vhi, self.nv))

    @property
    def cells(self) -> int:
        return int(np.prod(self.n)) * int(np.prod(self.nv))

    @property
    def shape(self) -> Tuple[int, ...]:
        return tuple(self.n) + tuple(self.nv)

    def centres_x(self, axis: int) -> np.ndarray:
        return self.box_lo[axis] + (np.arange(self.n[axis]) + 0.5) * self.dx[axis]

    def centres_v(self, axis: int) -> np.ndarray:
        return self.vlo[axis] + (np.arange(self.nv[axis]) + 0.5) * self.dv[axis]

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------------------
# seeded mode parameters
# ---------------------------------------------------------------------------

def random_modes(seed: int, count: int, nmax: float, amp: float = 1e-3,
                 nmin: float = 1.0):
    """Draw `count` Fourier modes with integer wave vectors n, nmin <= |n| <=
    nmax, amplitudes A ~ U[0, amp) and phases theta ~ U[0, 2 pi), from numpy's
    PCG64 generator seeded with `seed`."""
    rng = np.random.default_rng(seed)
    out = []
    lim = int(math.floor(nmax))
    while len(out) < count:
        nvec = tuple(int(t) for t in rng.integers(-lim, lim + 1, size=3))
        norm = math.sqrt(sum(t * t for t in nvec))
        if norm < nmin or norm > nmax:
            continue
        a = float(rng.uniform(0.0, amp))
        th = float(rng.uniform(0.0, 2.0 * math.pi))
        out.append((nvec, a, th))
    return tuple(out)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def _jeans_rho_bar(k_over_kj: float, k: float, sigma: float, G: float) -> float:
    """rho_bar that puts a mode of wave number k at k/k_J (Eq. jeans_wavenumber)."""
    kj = k / k_over_kj
    return kj * kj * sigma * sigma / (4.0 * math.pi * G)


def landau_c1() -> Workload:
    """Gravitational Landau damping, 16^3 x 16^3, FP64 storage, 20 steps."""
    L = 1.0
    return Workload(
        name="landau16_f64", n=(16, 16, 16), nv=(16, 16, 16),
        box_lo=(-L / 2,) * 3, box_hi=(L / 2,) * 3, vlo=(-5.0,) * 3, vhi=(5.0,) * 3,
        G=1.0, courant=0.5, dtype="f64", steps=20, seed=0,
        rho_bar=_jeans_rho_bar(1.5, 2 * math.pi / L, 1.0, 1.0), sigma=1.0,
        modes=(((1, 0, 0), 1e-2, 0.0),))


def jeans_c2() -> Workload:
    """Jeans instability, 32^3 x 32^3, FP32 f, 200 steps."""
    L = 1.0
    return Workload(
        name="jeans32_f32", n=(32, 32, 32), nv=(32, 32, 32),
        box_lo=(-L / 2,) * 3, box_hi=(L / 2,) * 3, vlo=(-5.0,) * 3, vhi=(5.0,) * 3,
        G=1.0, courant=0.5, dtype="f32", steps=200, seed=0,
        rho_bar=_jeans_rho_bar(0.5, 2 * math.pi / L, 1.0, 1.0), sigma=1.0,
        modes=(((1, 0, 0), 1e-3, 0.0),))


def king_c3(w0: float = 6.0, n: int = 64, nv: int = 32) -> Workload:
    """Isolated King sphere W0=6, 64^3 x 32^3, outflow boundaries, 300 steps.
    Units G = sigma = r0 = 1 with r0 = 3 sigma / sqrt(4 pi G rho_0).  The box
    half-width is 1.02 r_t and the velocity bound 3 sigma_c (central 1D
    dispersion)."""
    prof = king_profile(w0)
    half = 1.02 * prof.r_t
    vb = 3.0 * prof.sigma_c
    return Workload(
        name=f"king{n}x{nv}_w{w0:g}", n=(n,) * 3, nv=(nv,) * 3,
        box_lo=(-half,) * 3, box_hi=(half,) * 3, vlo=(-vb,) * 3, vhi=(vb,) * 3,
        G=1.0, courant=0.5, space_bc="outflow", poisson_bc="isolated",
        dtype="f32", steps=300, seed=0, ic="king", sigma=1.0, king_w0=w0)


def king_merger(w0: float = 3.0, nv: int = 32) -> Workload:
    """Two King spheres (W0 = 3) on the x axis, centres 2.2 r_t apart,
    approaching each other at 0.5 sigma_c each (the Vlasov side of the merger
    runs of Sec. 3.6).  64 x 32 x 32 cubic cells over a box of half-widths
    (2.15 r_t, 1.075 r_t, 1.075 r_t), velocities within 3 sigma_c + u,
    isolated Poisson, outflow boundaries, FP32."""
    prof = king_profile(w0)
    sep = 2.2 * prof.r_t
    u = 0.5 * prof.sigma_c
    hx, hy = 2.15 * prof.r_t, 1.075 * prof.r_t
    vb = 3.0 * prof.sigma_c + u
    return Workload(
        name=f"king_merger_w{w0:g}", n=(64, 32, 32), nv=(nv,) * 3,
        box_lo=(-hx, -hy, -hy), box_hi=(hx, hy, hy), vlo=(-vb,) * 3, vhi=(vb,) * 3,
        G=1.0, courant=0.5, space_bc="outflow", poisson_bc="isolated",
        dtype="f32", steps=200, seed=0, ic="king2", sigma=1.0, king_w0=w0,
        king_sep=sep, king_u=u)


def adjoint_c4() -> Workload:
    """Jeans setup with 3 random modes (seed 1), 100 steps, fixed dt."""
    L = 1.0
    return Workload(
        name="jeans32_modes3", n=(32, 32, 32), nv=(32, 32, 32),
        box_lo=(-L / 2,) * 3, box_hi=(L / 2,) * 3, vlo=(-5.0,) * 3, vhi=(5.0,) * 3,
        G=1.0, courant=0.5, dt_fixed=0.5 * (L / 32) / 5.0, dtype="f32",
        steps=100, seed=1, rho_bar=4 * math.pi, sigma=1.0,
        modes=random_modes(1, 3, 3.0))


def large_c5() -> Workload:
    """48^3 x 48^3 periodic Jeans box with 8 random modes (seed 2), 500 steps."""
    L = 1.0
    return Workload(
        name="jeans48_modes8", n=(48, 48, 48), nv=(48, 48, 48),
        box_lo=(-L / 2,) * 3, box_hi=(L / 2,) * 3, vlo=(-5.0,) * 3, vhi=(5.0,) * 3,
        G=1.0, courant=0.5, dt_fixed=0.5 * (L / 48) / 5.0, dtype="f32",
        steps=500, seed=2, rho_bar=4 * math.pi, sigma=1.0,
        modes=random_modes(2, 8, 4.0, nmin=0.6))


def small_maxwell(n=(8, 6, 5), nv=(12, 10, 9), dtype="f64", seed=3,
                  nmodes=3, amp=0.2, **kw) -> Workload:
    """A small, deliberately ragged Maxwellian box for parity tests."""
    L = 1.0
    base = dict(
        name=f"small{n}x{nv}", n=tuple(n), nv=tuple(nv),
        box_lo=(-L / 2, -0.6, -0.45), box_hi=(L / 2, 0.6, 0.45),
        vlo=(-4.0, -3.5, -4.5), vhi=(4.0, 4.5, 3.5),
        G=1.0, courant=0.5, dtype=dtype, steps=3, seed=seed,
        rho_bar=4 * math.pi, sigma=1.0, modes=random_modes(seed, nmodes, 2.0, amp=amp))
    base.update(kw)
    return Workload(**base)


def jeans_profile() -> Workload:
    """The 32^3-velocity Jeans set-up on a 16^3 spatial grid (537 MB of FP32 f,
    above the 129 MB L2): the same kernels as the 32^3 x 32^3 workload at an
    eighth of the size, for hardware-counter captures."""
    return jeans_c2().replace(name="jeans16x32_f32", n=(16, 16, 16))


def white_noise32(kj_over_k1: float = 4.0) -> Workload:
    """Test 4 (Sec. 3.4): 32^3 x 32^3 FP32 periodic box (L = 1, G = 1,
    sigma = 1, v in [-5, 5]^3) with a white-noise density contrast of rms
    1e-4 (seed 4); rho_bar sets the Jeans wavenumber k_J = kj_over_k1 * 2 pi / L
    (4: k_J = 8 pi / L, 8: 16 pi / L)."""
    L, sigma = 1.0, 1.0
    kj = kj_over_k1 * 2 * math.pi / L
    return Workload(
        name="white_noise32_kj%d" % int(kj_over_k1), n=(32, 32, 32), nv=(32, 32, 32),
        box_lo=(-L / 2,) * 3, box_hi=(L / 2,) * 3, vlo=(-5.0,) * 3, vhi=(5.0,) * 3,
        G=1.0, courant=0.5, dtype="f32", steps=200, seed=4, ic="noise",
        rho_bar=kj * kj * sigma * sigma / (4 * math.pi), sigma=sigma, noise_amp=1e-4)


def jeans_slab_yz() -> Workload:
    """A 4-plane slab (4 x 32 x 32 spatial cells) of the 32^3 x 32^3 Jeans
    box: the fused z + y drift at its full-size line length 32, with 537 MB
    of FP32 f (above L2), for hardware-counter captures."""
    return jeans_c2().replace(name="jeans_slab_yz_f32", n=(4, 32, 32))


def jeans_slab_x() -> Workload:
    """A 32 x 8 x 8 slab of the 32^3 x 32^3 Jeans box: the x drift with the
    fused density at line length 32, 268 MB of FP32 f (above L2)."""
    return jeans_c2().replace(name="jeans_slab_x_f32", n=(32, 8, 8))


def jeans48_slab() -> Workload:
    """8^3 spatial cells of the 48^3 x 48^3 box (226 MB of FP32 f, above L2):
    the 48^3-cube kick kernels for hardware-counter captures."""
    return large_c5().replace(name="jeans48_slab_f32", n=(8, 8, 8))


def adjoint_profile() -> Workload:
    """The fixed-dt 3-mode Jeans set-up on 16^3 positions (537 MB of FP32 f):
    the adjoint kernels of the 32^3 x 32^3 adjoint workload at line and cube
    length 32 (x lines 16), for hardware-counter captures."""
    return adjoint_c4().replace(name="jeans16x32_modes3", n=(16, 16, 16))


WORKLOADS = {
    "jeans16x32_f32": jeans_profile,
    "jeans16x32_modes3": adjoint_profile,
    "jeans48_slab_f32": jeans48_slab,
    "jeans_slab_yz_f32": jeans_slab_yz,
    "jeans_slab_x_f32": jeans_slab_x,
    "landau16_f64": landau_c1,
    "jeans32_f32": jeans_c2,
    "king64x32_w6": king_c3,
    "jeans32_modes3": adjoint_c4,
    "jeans48_modes8": large_c5,
    "white_noise32_kj4": white_noise32,
    "king_merger_w3": king_merger,
}


# ---------------------------------------------------------------------------
# initial conditions
# ---------------------------------------------------------------------------

def mode_fields(w: Workload) -> np.ndarray:
    """cos(k_m . x + theta_m) on the spatial cell centres, one 3D field per
    mode (shape (M, Nx, Ny, Nz)), k_m = 2 pi n_m / L."""
    L = [h - l for l, h in zip(w.box_lo, w.box_hi)]
    xs = [w.centres_x(a) for a in range(3)]
    out = np.empty((len(w.modes),) + tuple(w.n))
    for i, (nvec, _a, th) in enumerate(w.modes):
        ph = (2 * math.pi * nvec[0] / L[0] * xs[0][:, None, None]
              + 2 * math.pi * nvec[1] / L[1] * xs[1][None, :, None]
              + 2 * math.pi * nvec[2] / L[2] * xs[2][None, None, :])
        out[i] = np.cos(ph + th)
    return out


def density_contrast(w: Workload, amplitudes: Optional[Sequence[float]] = None) -> np.ndarray:
    """delta(x) = sum_m A_m cos(k_m . x + theta_m) on the spatial centres, or
    for ic "noise" white noise: independent Gaussian cell values of rms
    noise_amp (seeded PCG64), with their mean removed."""
    if w.ic == "noise":
        d = np.random.default_rng(w.seed).normal(0.0, w.noise_amp, size=w.n)
        return d - d.mean()
    if not w.modes:
        return np.zeros(w.n)
    amps = [m[1] for m in w.modes] if amplitudes is None else list(amplitudes)
    fields = mode_fields(w)
    return np.tensordot(np.asarray(amps, dtype=np.float64), fields, axes=1)


def maxwellian_v(w: Workload) -> np.ndarray:
    """(2 pi sigma^2)^{-3/2} exp(-|v|^2 / 2 sigma^2) on the velocity centres,
    shape (Nvx, Nvy, Nvz)."""
    s2 = w.sigma ** 2
    vx, vy, vz = (w.centres_v(a) for a in range(3))
    e = (np.exp(-vx ** 2 / (2 * s2))[:, None, None]
         * np.exp(-vy ** 2 / (2 * s2))[None, :, None]
         * np.exp(-vz ** 2 / (2 * s2))[None, None, :])
    return e * (2 * math.pi * s2) ** -1.5


def factors(w: Workload, amplitudes=None):
    """The Maxwellian initial condition as an outer product f = rho(x) M(v):
    (rho on the spatial centres, flat; M on the velocity centres, flat), both
    FP64.  The product of the two, rounded once, is initial_condition()."""
    rho_x = w.rho_bar * (1.0 + density_contrast(w, amplitudes))
    return rho_x.reshape(-1), maxwellian_v(w).reshape(-1)


def initial_condition(w: Workload, dtype=None, amplitudes=None) -> np.ndarray:
    """f(x, v, t=0) on the cell centres, C order [x][y][z][vx][vy][vz].
    Computed in FP64 and rounded once to the storage type."""
    dt = np.dtype(dtype or ("float32" if w.dtype == "f32" else "float64"))
    if w.ic in ("king", "king2"):
        return king_initial_condition(w, dt)
    rho_x, mv = factors(w, amplitudes)
    out = np.empty((int(np.prod(w.n)), mv.size), dtype=dt)
    flat = rho_x
    step = max(1, (1 << 24) // mv.size)
    for s in range(0, flat.size, step):
        e = min(flat.size, s + step)
        out[s:e] = np.multiply.outer(flat[s:e], mv).astype(dt)
    return out.reshape(w.shape)


def top_hat_1d(nx: int = 128, nv: int = 128, L: float = 1.0, vm: float = 1.0):
    """Test 1 (Sec. 3.1): f = 1 for |x| <= L/4 and |v| <= Vm/2, else 0, on a
    periodic [-L/2, L/2) x [-Vm, Vm] grid of cell centres.  Returns
    (f[x][v], x centres, v centres)."""
    x = -L / 2 + (np.arange(nx) + 0.5) * (L / nx)
    v = -vm + (np.arange(nv) + 0.5) * (2 * vm / nv)
    f = ((np.abs(x)[:, None] <= L / 4) & (np.abs(v)[None, :] <= vm / 2)).astype(np.float64)
    return f, x, v


# ---------------------------------------------------------------------------
# King sphere (Sec. 3.5)
# ---------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class KingProfile:
    w0: float
    r: np.ndarray        # radii in units of r0
    W: np.ndarray        # Psi / sigma^2 at r
    r_t: float           # tidal radius (W = 0)
    rho0: float          # central density (G = sigma = r0 = 1)
    rho1: float          # DF normalisation rho_1
    sigma_c: float       # central 1D velocity dispersion

    def psi(self, radius: np.ndarray) -> np.ndarray:
        """Psi(r) / sigma^2, 0 beyond r_t (f vanishes there)."""
        out = np.interp(radius, self.r, self.W, right=0.0)
        return np.where(radius >= self.r_t, 0.0, out)


def _king_density(W):
    """rho(Psi)/rho_1 for the lowered isothermal DF, W = Psi/sigma^2."""
    from scipy.special import erf
    W = np.maximum(W, 0.0)
    return np.exp(W) * erf(np.sqrt(W)) - np.sqrt(4 * W / math.pi) * (1 + 2 * W / 3)


def _trapz(y, x):
    return float(np.sum(0.5 * (y[1:] + y[:-1]) * np.diff(x)))


def king_profile(w0: float = 6.0) -> KingProfile:
    """Integrate the King ODE  W'' + 2 W'/r = -9 rho(W)/rho(W0)  (r in units of
    r0 = 3 sigma / sqrt(4 pi G rho_0)) from W(0) = W0 to W(r_t) = 0."""
    from scipy.integrate import solve_ivp
    from scipy.special import erf
    rho_w0 = float(_king_density(np.array(w0)))

    def rhs(r, y):
        W, dW = y
        return [dW, -9.0 * float(_king_density(np.array(W))) / rho_w0 - 2.0 * dW / r]

    r_start = 1e-6
    y0 = [w0 - 1.5 * r_start ** 2, -3.0 * r_start]

    def hit_zero(r, y):
        return y[0]
    hit_zero.terminal = True
    hit_zero.direction = -1
    sol = solve_ivp(rhs, (r_start, 1e4), y0, events=hit_zero, rtol=1e-11, atol=1e-13,
                    dense_output=True, method="DOP853")
    r_t = float(sol.t_events[0][0])
    r = np.concatenate([[0.0], np.linspace(r_start, r_t, 20001)])
    W = np.concatenate([[w0], sol.sol(r[1:])[0]])
    W[-1] = 0.0
    rho0 = 9.0 / (4.0 * math.pi)           # G = sigma = r0 = 1
    rho1 = rho0 / rho_w0
    # central 1D dispersion: <v_x^2> = (integral f v^4 dv) / (3 integral f v^2 dv) at Psi = W0
    v = np.linspace(0.0, math.sqrt(2 * w0), 200001)
    fv = np.exp(w0 - v * v / 2) - 1.0
    num = _trapz(fv * v ** 4, v)
    den = _trapz(fv * v ** 2, v)
    sigma_c = math.sqrt(num / (3 * den))
    del erf
    return KingProfile(w0=w0, r=r, W=W, r_t=r_t, rho0=rho0, rho1=rho1, sigma_c=sigma_c)


def king_factors(w: Workload):
    """The pieces of the King DF at the cell centres: per sphere the relative
    potential Psi on the spatial centres (flat) and |v - u|^2 on the velocity
    centres (flat), and the normalisation; f = norm sum_spheres
    expm1(Psi - |v - u|^2 / 2) where that is positive (sigma = 1)."""
    prof = king_profile(w.king_w0)
    xs = [w.centres_x(a) for a in range(3)]
    vx, vy, vz = (w.centres_v(a) for a in range(3))
    norm = prof.rho1 * (2 * math.pi) ** -1.5
    if w.ic == "king2":
        spheres = ((-0.5 * w.king_sep, w.king_u), (0.5 * w.king_sep, -w.king_u))
    else:
        spheres = ((0.0, 0.0),)
    psis, v2s = [], []
    for cx, ux in spheres:
        r = np.sqrt((xs[0][:, None, None] - cx) ** 2 + xs[1][None, :, None] ** 2
                    + xs[2][None, None, :] ** 2)
        psis.append(prof.psi(r).reshape(-1))             # sigma = 1
        v2s.append(((vx - ux)[:, None, None] ** 2 + vy[None, :, None] ** 2
                    + vz[None, None, :] ** 2).reshape(-1))
    return psis, v2s, norm


def king_initial_condition_device(w: Workload, device, dtype):
    """king_initial_condition() evaluated in FP64 on a torch device from the
    same factors (rounded once to dtype; expm1 is the device's, so a value
    can differ from the host evaluation in its last FP64 bit)."""
    import torch
    psis, v2s, norm = king_factors(w)
    npos, nvel = psis[0].size, v2s[0].size
    out = torch.empty((npos, nvel), dtype=dtype, device=device)
    ps = [torch.from_numpy(p).to(device) for p in psis]
    vs = [torch.from_numpy(v).to(device) for v in v2s]
    step = max(1, (1 << 26) // nvel)
    for s in range(0, npos, step):
        e = min(npos, s + step)
        acc = torch.zeros((e - s, nvel), dtype=torch.float64, device=device)
        for p, v in zip(ps, vs):
            E = p[s:e, None] - 0.5 * v[None, :]
            acc += torch.where(E > 0, torch.expm1(torch.clamp(E, min=0.0)), torch.zeros_like(E))
        out[s:e] = (norm * acc).to(dtype)
    return out.reshape(w.shape)


def king_initial_condition(w: Workload, dtype) -> np.ndarray:
    """King DF at the cell centres, before the virial renormalisation; for
    ic "king2" the sum of two King spheres centred at x = -+ king_sep / 2 and
    moving at v_x = +- king_u (towards each other)."""
    psis, v2s, norm = king_factors(w)
    npos, nvel = psis[0].size, v2s[0].size
    out = np.empty((npos, nvel), dtype=dtype)
    step = max(1, (1 << 24) // nvel)
    for s in range(0, npos, step):
        e = min(npos, s + step)
        acc = np.zeros((e - s, nvel))
        for psi, v2 in zip(psis, v2s):
            E = psi[s:e, None] - 0.5 * v2[None, :]
            acc += np.where(E > 0, np.expm1(np.maximum(E, 0.0)), 0.0)
        out[s:e] = (norm * acc).astype(dtype)
    return out.reshape(w.shape)
