"""The Python binding refuses tensors the library cannot take (wrong device,
dtype, shape or memory layout) before any pointer reaches the C ABI: the
library dereferences them on the GPU.  Checked on a stand-in object with f
on the host and a recording library (no CUDA needed): valid arguments reach
the library, invalid ones raise ValueError and reach nothing."""
import ctypes

import pytest
import torch

from paper_1206_6152_gb300.vlasov import VlasovPoisson, make_config

N, NV = (4, 3, 2), (5, 4, 3)


class Recorder:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            return 0
        return call


def stand_in(dtype=torch.float64):
    sim = VlasovPoisson.__new__(VlasovPoisson)
    sim.cfg = make_config(N, NV, (0.0,) * 3, (1.0,) * 3, (-1.0,) * 3, (1.0,) * 3, dtype=dtype)
    sim.f = torch.zeros(N + NV, dtype=dtype)
    sim.device = sim.f.device
    sim._ctx = ctypes.c_void_p()
    sim.lib = Recorder()
    return sim


def f_like(sim, **kw):
    return torch.zeros(N + NV, dtype=kw.get("dtype", sim.f.dtype), device=kw.get("device", "cpu"))


def g_like(k=3, **kw):
    shape = N if k == 1 else (k,) + N
    return torch.zeros(shape, dtype=kw.get("dtype", torch.float64), device=kw.get("device", "cpu"))


def test_valid_arguments_reach_the_library():
    sim = stand_in()
    sim.adjoint_step(f_like(sim), g_like(), f_like(sim), g_like())
    sim.sweep_adjoint(3, 0.1, f_like(sim), f_like(sim), g_like())
    sim.sweep_adjoint(0, 0.1, f_like(sim), f_like(sim))
    sim.field_adjoint(g_like(), f_like(sim))
    sim.functional(0, f_like(sim))
    sim.functional(1, f_like(sim), g_like(1))
    sim.set_accel(g_like())
    sim.set_distribution(f_like(sim))
    sim.step_host(f_like(sim), 1, f_like(sim))
    assert sim.lib.calls == ["vp_adjoint_step", "vp_sweep_adjoint", "vp_sweep_adjoint",
                             "vp_field_adjoint", "vp_functional", "vp_functional", "vp_set_accel",
                             "vp_set_distribution", "vp_step_host"]


@pytest.mark.parametrize("bad", ["dtype", "shape", "layout", "device"])
def test_invalid_state_tensors_are_refused(bad):
    sim = stand_in()
    if bad == "dtype":
        x = f_like(sim, dtype=torch.float32)
    elif bad == "shape":
        x = torch.zeros((2,) + N + NV, dtype=torch.float64)[0].reshape(N[::-1] + NV)
    elif bad == "layout":
        x = torch.zeros(N + NV[::-1], dtype=torch.float64).permute(0, 1, 2, 5, 4, 3)
    else:
        x = f_like(sim, device="meta")
    calls = [
        lambda: sim.adjoint_step(x, g_like(), f_like(sim), g_like()),
        lambda: sim.adjoint_step(f_like(sim), g_like(), x, g_like()),
        lambda: sim.sweep_adjoint(3, 0.1, x, f_like(sim)),
        lambda: sim.sweep_adjoint(3, 0.1, f_like(sim), x),
        lambda: sim.field_adjoint(g_like(), x),
        lambda: sim.functional(0, x),
        lambda: sim.set_distribution(x),
    ]
    for c in calls:
        with pytest.raises(ValueError):
            c()
    assert sim.lib.calls == []


@pytest.mark.parametrize("bad", ["dtype", "shape", "device"])
def test_invalid_field_tensors_are_refused(bad):
    sim = stand_in()
    if bad == "dtype":
        g3, g1 = g_like(dtype=torch.float32), g_like(1, dtype=torch.float32)
    elif bad == "shape":
        g3, g1 = g_like(2), torch.zeros(N[::-1], dtype=torch.float64)
    else:
        g3, g1 = g_like(device="meta"), g_like(1, device="meta")
    calls = [
        lambda: sim.adjoint_step(f_like(sim), g3, f_like(sim), g_like()),
        lambda: sim.adjoint_step(f_like(sim), g_like(), f_like(sim), g3),
        lambda: sim.sweep_adjoint(3, 0.1, f_like(sim), f_like(sim), g3),
        lambda: sim.field_adjoint(g3, f_like(sim)),
        lambda: sim.functional(1, f_like(sim), g1),
    ]
    if bad == "shape":
        calls.append(lambda: sim.set_accel(g3))
    for c in calls:
        with pytest.raises(ValueError):
            c()
    assert sim.lib.calls == []


def test_host_buffers_must_be_host_tensors_of_f():
    sim = stand_in(torch.float32)
    for x in (f_like(sim, dtype=torch.float64), f_like(sim, device="meta"),
              torch.zeros((1,) + N + NV, dtype=torch.float32)):
        with pytest.raises(ValueError):
            sim.step_host(x, 1)
        with pytest.raises(ValueError):
            sim.step_host(f_like(sim), 1, x)
    assert sim.lib.calls == []
