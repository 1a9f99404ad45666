"""Python front end of the C ABI (include/vp.h).

PyTorch supplies the device memory and the stream; every step of the
computation runs in the library's CUDA kernels.  A VlasovPoisson object
borrows a torch tensor f of shape (Nx, Ny, Nz, Nvx, Nvy, Nvz) on the current
CUDA device and advances it in place.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

import torch

from . import _lib
from ._lib import check, vp_config

_DTYPES = {torch.float32: 0, torch.float64: 1}


def make_config(n, nv, box_lo, box_hi, vlo, vhi, G=1.0, courant=0.5, dt_fixed=0.0,
                space_bc="periodic", poisson_bc="periodic", dtype=torch.float32) -> vp_config:
    c = vp_config()
    for a in range(3):
        c.n[a] = int(n[a])
        c.nv[a] = int(nv[a])
        c.box_lo[a] = float(box_lo[a])
        c.box_hi[a] = float(box_hi[a])
        c.vlo[a] = float(vlo[a])
        c.vhi[a] = float(vhi[a])
    c.G = float(G)
    c.courant = float(courant)
    c.dt_fixed = float(dt_fixed)
    c.space_bc = {"periodic": 0, "outflow": 1}[space_bc]
    c.poisson_bc = {"periodic": 0, "isolated": 1}[poisson_bc]
    c.dtype = _DTYPES[dtype]
    return c


def config_of(workload, dtype=None) -> vp_config:
    """vp_config of an inputs.Workload."""
    dt = dtype or (torch.float32 if workload.dtype == "f32" else torch.float64)
    return make_config(workload.n, workload.nv, workload.box_lo, workload.box_hi, workload.vlo,
                       workload.vhi, workload.G, workload.courant, workload.dt_fixed,
                       workload.space_bc, workload.poisson_bc, dt)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class VlasovPoisson:
    """One 6D Vlasov--Poisson system on one GPU (see include/vp.h)."""

    def __init__(self, cfg: vp_config, f: torch.Tensor, stream: Optional[torch.cuda.Stream] = None):
        if not f.is_cuda or not f.is_contiguous():
            raise ValueError("f must be a contiguous CUDA tensor")
        shape = tuple(cfg.n) + tuple(cfg.nv)
        if tuple(f.shape) != shape:
            raise ValueError(f"f has shape {tuple(f.shape)}, expected {shape}")
        if _DTYPES.get(f.dtype) != cfg.dtype:
            raise ValueError("f dtype does not match the configuration")
        self.lib = _lib.load()
        self.cfg = cfg
        self.f = f
        self.device = f.device
        self.stream = stream or torch.cuda.current_stream(f.device)
        self.np = int(cfg.n[0] * cfg.n[1] * cfg.n[2])
        self._ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.vp_init(ctypes.byref(cfg), _ptr(f), ctypes.c_void_p(self.stream.cuda_stream),
                                   ctypes.byref(self._ctx)), "vp_init")

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if self._ctx:
            self.lib.vp_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- stepping ---------------------------------------------------------
    def step(self, nsteps: int = 1, sync: bool = False) -> Optional[float]:
        t = ctypes.c_double()
        check(self.lib.vp_step(self._ctx, int(nsteps), ctypes.byref(t) if sync else None), "vp_step")
        return t.value if sync else None

    def sweep(self, axis: int, tau: float) -> None:
        check(self.lib.vp_sweep(self._ctx, int(axis), float(tau)), "vp_sweep")

    # -- argument checks: the library dereferences the pointers on the GPU,
    # so a tensor of the wrong kind is refused here rather than read there
    def _state(self, t: torch.Tensor, name: str) -> torch.Tensor:
        """A contiguous tensor of f's shape and dtype on f's device."""
        if (not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != self.f.dtype
                or tuple(t.shape) != tuple(self.f.shape) or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous {self.f.dtype} tensor of shape "
                             f"{tuple(self.f.shape)} on {self.device}")
        return t

    def _host_state(self, t: torch.Tensor, name: str) -> torch.Tensor:
        """A contiguous host tensor of f's shape and dtype."""
        if (not isinstance(t, torch.Tensor) or t.device.type != "cpu" or t.dtype != self.f.dtype
                or tuple(t.shape) != tuple(self.f.shape) or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous host {self.f.dtype} tensor of shape "
                             f"{tuple(self.f.shape)}")
        return t

    def _field_arg(self, t: torch.Tensor, k: int, name: str) -> torch.Tensor:
        """A contiguous float64 tensor of shape (k, Nx, Ny, Nz) (k = 1: (Nx, Ny, Nz))
        on f's device."""
        n = tuple(self.cfg.n)
        shape = n if k == 1 else (k,) + n
        if (not isinstance(t, torch.Tensor) or t.device != self.device
                or t.dtype != torch.float64 or tuple(t.shape) != shape or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float64 tensor of shape {shape} on "
                             f"{self.device}")
        return t

    def set_distribution(self, f: torch.Tensor) -> None:
        self._state(f, "f")
        check(self.lib.vp_set_distribution(self._ctx, _ptr(f)), "vp_set_distribution")
        self.f = f

    def refresh_field(self) -> None:
        check(self.lib.vp_refresh_field(self._ctx), "vp_refresh_field")

    # -- fields and diagnostics ------------------------------------------
    def _spatial(self, k=1):
        n = tuple(self.cfg.n)
        return torch.empty((k,) + n if k > 1 else n, dtype=torch.float64, device=self.device)

    def density(self) -> torch.Tensor:
        rho = self._spatial()
        check(self.lib.vp_moments(self._ctx, _ptr(rho)), "vp_moments")
        return rho

    def field(self) -> Tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
        rho, phi, g = self._spatial(), self._spatial(), self._spatial(3)
        check(self.lib.vp_get_field(self._ctx, _ptr(rho), _ptr(phi), _ptr(g)), "vp_get_field")
        return rho, phi, g

    def set_accel(self, g: torch.Tensor) -> None:
        g = self._field_arg(g.to(device=self.device, dtype=torch.float64).contiguous(), 3, "g")
        check(self.lib.vp_set_accel(self._ctx, _ptr(g)), "vp_set_accel")
        self._keep = g

    def energy(self) -> dict:
        out = (ctypes.c_double * 5)()
        check(self.lib.vp_energy(self._ctx, out), "vp_energy")
        return dict(M=out[0], K=out[1], U=out[2], E=out[3], M_out=out[4])

    def time(self) -> Tuple[float, float]:
        t, dt = ctypes.c_double(), ctypes.c_double()
        check(self.lib.vp_time(self._ctx, ctypes.byref(t), ctypes.byref(dt)), "vp_time")
        return t.value, dt.value

    def step_host(self, f_host_in: torch.Tensor, nsteps: int, f_host_out: Optional[torch.Tensor] = None,
                  diagnostics: bool = False):
        self._host_state(f_host_in, "f_host_in")
        if f_host_out is not None:
            self._host_state(f_host_out, "f_host_out")
        t = ctypes.c_double()
        diag = (ctypes.c_double * 5)() if diagnostics else None
        check(self.lib.vp_step_host(self._ctx, _ptr(f_host_in), _ptr(f_host_out), int(nsteps),
                                    ctypes.byref(t), diag), "vp_step_host")
        return t.value, (list(diag) if diag is not None else None)

    # -- tracing ----------------------------------------------------------
    def profile_step(self) -> dict:
        out = (ctypes.c_double * _lib.PROFILE_SLOTS)()
        check(self.lib.vp_profile_step(self._ctx, out), "vp_profile_step")
        return dict(zip(_lib.PROFILE_NAMES, list(out)))

    def check(self) -> Tuple[int, int]:
        """(cells of f that are NaN or infinite, cells below zero)."""
        out = (ctypes.c_longlong * 2)()
        code = self.lib.vp_check(self._ctx, out)
        if code not in (0, -4):
            check(code, "vp_check")
        return int(out[0]), int(out[1])

    def kernels_launched(self) -> int:
        n = ctypes.c_longlong()
        check(self.lib.vp_stats(self._ctx, ctypes.byref(n)), "vp_stats")
        return n.value

    # -- adjoint ----------------------------------------------------------
    def adjoint_step(self, f_start: torch.Tensor, g_start: torch.Tensor, lam_f: torch.Tensor,
                     lam_g: torch.Tensor) -> None:
        self._state(f_start, "f_start")
        self._field_arg(g_start, 3, "g_start")
        self._state(lam_f, "lam_f")
        self._field_arg(lam_g, 3, "lam_g")
        check(self.lib.vp_adjoint_step(self._ctx, _ptr(f_start), _ptr(g_start), _ptr(lam_f),
                                       _ptr(lam_g)), "vp_adjoint_step")

    def set_adjoint_states(self, mode: int) -> None:
        """Scratch policy of adjoint_step: 0 automatic, 1 two states
        (recompute), 2 the kept sweep inputs (at most eight states), 3 three
        states."""
        check(self.lib.vp_set_adjoint_states(self._ctx, int(mode)), "vp_set_adjoint_states")

    def sweep_adjoint(self, axis: int, tau: float, f_in: torch.Tensor, lam: torch.Tensor,
                      lam_g: Optional[torch.Tensor] = None) -> None:
        self._state(f_in, "f_in")
        self._state(lam, "lam")
        if lam_g is not None:
            self._field_arg(lam_g, 3, "lam_g")
        check(self.lib.vp_sweep_adjoint(self._ctx, int(axis), float(tau), _ptr(f_in), _ptr(lam),
                                        _ptr(lam_g)), "vp_sweep_adjoint")

    def field_adjoint(self, lam_g: torch.Tensor, lam_f: torch.Tensor) -> None:
        self._field_arg(lam_g, 3, "lam_g")
        self._state(lam_f, "lam_f")
        check(self.lib.vp_field_adjoint(self._ctx, _ptr(lam_g), _ptr(lam_f)), "vp_field_adjoint")

    def functional(self, kind: int, lam_f: torch.Tensor, target: Optional[torch.Tensor] = None) -> float:
        self._state(lam_f, "lam_f")
        if target is not None:
            self._field_arg(target, 1, "target")
        J = ctypes.c_double()
        check(self.lib.vp_functional(self._ctx, int(kind), _ptr(target), _ptr(lam_f), ctypes.byref(J)),
              "vp_functional")
        return J.value
