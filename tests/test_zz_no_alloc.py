"""The allocation-free moments entry point (vp_moments_noalloc) against the
context-based diagnostics (vp_energy) and the FP64 oracle's M and K on the
same f, called twice in a row with different inputs (the second time on
another stream, after the first has finished), through the C ABI; host
pointers are refused before anything is launched.

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

from oracle import vp_oracle as O  # noqa: E402
from paper_1206_6152_gb300 import inputs as I  # noqa: E402


def _call(lib, f, w, dtype_code, sums, stream):
    n = (ctypes.c_int * 3)(*w.n)
    nv = (ctypes.c_int * 3)(*w.nv)
    vlo = (ctypes.c_double * 3)(*w.vlo)
    vhi = (ctypes.c_double * 3)(*w.vhi)
    return lib.vp_moments_noalloc(ctypes.c_void_p(f.data_ptr()), dtype_code, n, nv, vlo, vhi,
                                  ctypes.c_void_p(sums.data_ptr()),
                                  ctypes.c_void_p(stream.cuda_stream) if stream is not None else None)


def _noalloc(lib, f, w, dtype_code, stream):
    sums = torch.zeros(2, dtype=torch.float64, device=f.device)
    rc = _call(lib, f, w, dtype_code, sums, stream)
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
    tdt = torch.float32 if dtype == "f32" else torch.float64
    code = 0 if dtype == "f32" else 1
    # two calls in a row with different grids and data, the second on
    # another stream once the first has finished: the second must not see
    # anything the first left in the shared scratch
    streams = [torch.cuda.current_stream(), torch.cuda.Stream()]
    for k, w in enumerate([I.small_maxwell(n=(16, 8, 12), nv=(10, 8, 12), dtype=dtype, amp=0.3),
                           I.small_maxwell(n=(6, 5, 4), nv=(12, 10, 9), dtype=dtype, amp=0.1,
                                           seed=7)]):
        f_np = (I.initial_condition(w) * (1.0 + 0.5 * k)).astype(np.float32 if dtype == "f32"
                                                                 else np.float64)
        f = torch.from_numpy(f_np).to("cuda:0", tdt)
        torch.cuda.synchronize()
        sums = _noalloc(lib, f, w, code, streams[k])
        with VlasovPoisson(config_of(w, tdt), f) as sim:
            e = sim.energy()
        dV = float(np.prod(w.dx)) * float(np.prod(w.dv))
        assert sums[0] * dV == pytest.approx(e["M"], rel=1e-13)
        assert 0.5 * sums[1] * dV == pytest.approx(e["K"], rel=1e-13)
        # the oracle's M and K (Sec. 3.1) of the same values
        M, K, _, _ = O.energy(f_np.astype(np.float64), O.Grid.of(w), O.Params(G=0.0))
        assert sums[0] * dV == pytest.approx(M, rel=1e-12)
        assert 0.5 * sums[1] * dV == pytest.approx(K, rel=1e-12)


@pytest.mark.gpu
def test_moments_noalloc_refuses_host_pointers():
    """A host buffer passed as f or as the output is refused with
    VP_ERR_ARG before any kernel runs."""
    from paper_1206_6152_gb300 import _lib
    lib = _lib.load()
    w = I.small_maxwell(n=(4, 4, 4), nv=(4, 4, 4), dtype="f32")
    f_host = torch.from_numpy(I.initial_condition(w))
    f_dev = f_host.to("cuda:0")
    sums_dev = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    sums_host = torch.zeros(2, dtype=torch.float64)
    assert _call(lib, f_host, w, 0, sums_dev, None) == -5
    assert _call(lib, f_dev, w, 0, sums_host, None) == -5
    assert _call(lib, f_host.pin_memory(), w, 0, sums_dev, None) == -5
    assert float(sums_dev.abs().sum()) == 0.0
    assert _call(lib, f_dev, w, 0, sums_dev, None) == 0
    torch.cuda.synchronize()
    assert float(sums_dev[0]) > 0.0


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
