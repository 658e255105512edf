"""GB300-native (sm_103a) distilled multi-time-step molecular dynamics.

Energy and force evaluation of two invariant message-passing potentials
(a 5.0 A "big" model and a distilled 3.5 A "small" model) and the RESPA
multiple-time-step integrator that combines them (Algorithm 1 of arXiv
2510.06562), as hand-written CUDA kernels behind a C ABI
(``include/dmts.h``, ``libdmts.so``).

``inputs`` draws seeded synthetic systems and parameters; ``dmts`` is the
ctypes binding of the C ABI (imported on first use so that the input
generators work without the compiled library).
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "dmts"]


def __getattr__(name):
    if name in ("dmts", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
