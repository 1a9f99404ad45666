"""GB300-native six-dimensional Vlasov--Poisson integrator (PFC split sweeps).

The computation lives in the CUDA library libvp.so (C ABI: include/vp.h);
`vlasov.VlasovPoisson` is its Python front end and `inputs` builds seeded
initial conditions.  Submodules are imported lazily so that the input
generator can be used without loading the CUDA library.
"""
import importlib

__all__ = ["inputs", "vlasov", "build", "adjoint"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
