"""ctypes binding of include/vp.h: argument marshalling only.

Every entry point of the C ABI appears here under the same name.  Nothing in
this module computes: it converts Python/torch arguments to pointers and
sizes and raises VPError on a negative status.  The library is loaded from the
package directory (built in-tree by build.py); if it is missing the import of
the binding fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvp.so")

# names the header declares, checked by the tests against the export table
EXPORTS = (
    "vp_init", "vp_set_distribution", "vp_refresh_field", "vp_step", "vp_sweep",
    "vp_moments", "vp_get_field", "vp_set_accel", "vp_energy", "vp_time", "vp_step_host",
    "vp_adjoint_step", "vp_field_adjoint", "vp_functional", "vp_destroy", "vp_error_string",
    "vp_profile_step", "vp_stats", "vp_sweep_adjoint", "vp_moments_noalloc",
    "vp_set_adjoint_states", "vp_check", "vp_debug_fail_alloc", "vp_line_max_x",
    "vp_drift_x_ghosted", "vp_field_init", "vp_field_solve", "vp_kick", "vp_drift_yz",
)
PROFILE_SLOTS = 11
PROFILE_NAMES = ("kick6", "drift_z", "drift_y", "drift_x", "density", "field", "tables", "step",
                 "kick_a", "kick_b", "kick_c")


class VPError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed with {code}: {msg}")
        self.code = code


class vp_config(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("nv", ctypes.c_int * 3),
        ("box_lo", ctypes.c_double * 3),
        ("box_hi", ctypes.c_double * 3),
        ("vlo", ctypes.c_double * 3),
        ("vhi", ctypes.c_double * 3),
        ("G", ctypes.c_double),
        ("courant", ctypes.c_double),
        ("dt_fixed", ctypes.c_double),
        ("space_bc", ctypes.c_int),
        ("poisson_bc", ctypes.c_int),
        ("dtype", ctypes.c_int),
    ]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libvp.so and declares the signatures.  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: run __graft_entry__.build() (or "
                              "python -m paper_1206_6152_gb300.build) first")
        L = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        i, d = ctypes.c_int, ctypes.c_double
        dp = ctypes.POINTER(ctypes.c_double)
        sig = {
            "vp_init": (i, [ctypes.POINTER(vp_config), vp, vp, ctypes.POINTER(vp)]),
            "vp_set_distribution": (i, [vp, vp]),
            "vp_refresh_field": (i, [vp]),
            "vp_step": (i, [vp, i, dp]),
            "vp_sweep": (i, [vp, i, d]),
            "vp_moments": (i, [vp, vp]),
            "vp_get_field": (i, [vp, vp, vp, vp]),
            "vp_set_accel": (i, [vp, vp]),
            "vp_energy": (i, [vp, dp]),
            "vp_time": (i, [vp, dp, dp]),
            "vp_step_host": (i, [vp, vp, vp, i, dp, dp]),
            "vp_adjoint_step": (i, [vp, vp, vp, vp, vp]),
            "vp_set_adjoint_states": (i, [vp, i]),
            "vp_field_adjoint": (i, [vp, vp, vp]),
            "vp_sweep_adjoint": (i, [vp, i, d, vp, vp, vp]),
            "vp_moments_noalloc": (i, [vp, i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       dp, dp, vp, vp]),
            "vp_functional": (i, [vp, i, vp, vp, dp]),
            "vp_destroy": (None, [vp]),
            "vp_error_string": (ctypes.c_char_p, [i]),
            "vp_profile_step": (i, [vp, dp]),
            "vp_stats": (i, [vp, ctypes.POINTER(ctypes.c_longlong)]),
            "vp_check": (i, [vp, ctypes.POINTER(ctypes.c_longlong)]),
            "vp_debug_fail_alloc": (i, [i]),
            "vp_line_max_x": (i, [vp, vp]),
            "vp_drift_x_ghosted": (i, [vp, d, vp, vp, i, vp]),
            "vp_field_init": (i, [ctypes.POINTER(vp_config), vp, ctypes.POINTER(vp)]),
            "vp_field_solve": (i, [vp, vp, vp, dp]),
            "vp_kick": (i, [vp, d, d]),
            "vp_drift_yz": (i, [vp, d]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def check(code: int, where: str) -> None:
    if code != 0:
        msg = load().vp_error_string(code)
        raise VPError(code, where, msg.decode() if msg else "?")
