"""CPU checks of the C ABI: the library builds, loads and exports every entry
point include/vp.h declares; argument and configuration checks that run on
the host before any CUDA call return the documented codes."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1206_6152_gb300 import build as B
    B.build()
    from paper_1206_6152_gb300 import _lib
    return _lib.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "vp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vp_[a-z_]+)\s*\(", text)))


def test_header_names_match_binding():
    from paper_1206_6152_gb300 import _lib
    assert header_functions() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_error_strings(lib):
    for code in (0, -1, -2, -4, -5, -6, -7):
        assert lib.vp_error_string(code)
    assert lib.vp_error_string(-99) == b"unknown error"


def _cfg(**kw):
    from paper_1206_6152_gb300.vlasov import make_config
    base = dict(n=(4, 4, 4), nv=(4, 4, 4), box_lo=(-0.5,) * 3, box_hi=(0.5,) * 3,
                vlo=(-1,) * 3, vhi=(1,) * 3)
    base.update(kw)
    return make_config(**base)


def test_null_arguments_rejected(lib):
    ctx = ctypes.c_void_p()
    assert lib.vp_init(None, ctypes.c_void_p(1), None, ctypes.byref(ctx)) == -5
    cfg = _cfg()
    assert lib.vp_init(ctypes.byref(cfg), None, None, ctypes.byref(ctx)) == -5
    assert lib.vp_step(None, 1, None) == -5
    assert lib.vp_energy(None, None) == -5
    assert lib.vp_sweep(None, 0, 0.1) == -5


@pytest.mark.parametrize("bad", [
    dict(n=(0, 4, 4)), dict(nv=(4, -1, 4)), dict(box_lo=(1, 0, 0), box_hi=(0, 1, 1)),
    dict(vlo=(1, 1, 1), vhi=(1, 1, 1)), dict(courant=0.0), dict(G=float("nan")),
])
def test_invalid_config_rejected_before_cuda(lib, bad):
    cfg = _cfg(**bad)
    ctx = ctypes.c_void_p()
    # a fake non-null pointer: the configuration check runs before any use
    assert lib.vp_init(ctypes.byref(cfg), ctypes.c_void_p(16), None, ctypes.byref(ctx)) == -1
    assert not ctx.value


def test_fault_injection_switch(lib):
    assert lib.vp_debug_fail_alloc(-1) == -5
    assert lib.vp_debug_fail_alloc(0) == 0
    assert lib.vp_check(None, None) == -5
