"""The allocation-free moments entry point (vp_moments_noalloc) against the
context-based diagnostics (vp_energy) on the same f, called twice in a row
with different inputs, through the C ABI.

Callers that cannot allocate device memory (inside a stream capture, or
under an allocator fixed at start-up) use vp_moments_noalloc, whose scratch
is a static device array of the library.  This file is collected last so a
failure here never hides the results of the other tests."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = pytest.mark.skip(reason="needs a CUDA GPU")

from paper_1206_6152_gb300 import inputs as I  # noqa: E402


def _noalloc(lib, f, w, dtype_code, stream):
    sums = torch.zeros(2, dtype=torch.float64, device=f.device)
    n = (ctypes.c_int * 3)(*w.n)
    nv = (ctypes.c_int * 3)(*w.nv)
    vlo = (ctypes.c_double * 3)(*w.vlo)
    vhi = (ctypes.c_double * 3)(*w.vhi)
    rc = lib.vp_moments_noalloc(ctypes.c_void_p(f.data_ptr()), dtype_code, n, nv, vlo, vhi,
                                ctypes.c_void_p(sums.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.vp_error_string(rc)
    torch.cuda.synchronize()
    return sums.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_moments_noalloc_matches_energy(dtype):
    from paper_1206_6152_gb300 import build as B
    B.build()
    from paper_1206_6152_gb300 import _lib
    from paper_1206_6152_gb300.vlasov import VlasovPoisson, config_of
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    tdt = torch.float32 if dtype == "f32" else torch.float64
    code = 0 if dtype == "f32" else 1
    # two calls in a row with different grids and data: the second must not
    # see anything the first left in the shared scratch
    for k, w in enumerate([I.small_maxwell(n=(16, 8, 12), nv=(10, 8, 12), dtype=dtype, amp=0.3),
                           I.small_maxwell(n=(6, 5, 4), nv=(12, 10, 9), dtype=dtype, amp=0.1,
                                           seed=7)]):
        f = torch.from_numpy(I.initial_condition(w) * (1.0 + 0.5 * k)).to("cuda:0", tdt)
        sums = _noalloc(lib, f, w, code, stream)
        with VlasovPoisson(config_of(w, tdt), f) as sim:
            e = sim.energy()
        dV = float(np.prod(w.dx)) * float(np.prod(w.dv))
        assert sums[0] * dV == pytest.approx(e["M"], rel=1e-13)
        assert 0.5 * sums[1] * dV == pytest.approx(e["K"], rel=1e-13)


@pytest.mark.gpu
def test_moments_noalloc_rejects_oversized_grid():
    from paper_1206_6152_gb300 import _lib
    lib = _lib.load()
    f = torch.zeros(8, dtype=torch.float32, device="cuda:0")
    sums = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    n = (ctypes.c_int * 3)(128, 64, 64)          # 2^19 spatial cells > 2^18
    nv = (ctypes.c_int * 3)(1, 1, 1)
    v0 = (ctypes.c_double * 3)(-1, -1, -1)
    v1 = (ctypes.c_double * 3)(1, 1, 1)
    rc = lib.vp_moments_noalloc(ctypes.c_void_p(f.data_ptr()), 0, n, nv, v0, v1,
                                ctypes.c_void_p(sums.data_ptr()), None)
    assert rc == -7
