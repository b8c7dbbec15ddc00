"""GB300-native circuit cutting for state-vector simulation.

The hot path (subcircuit simulation, merging, uncut simulation, FP64
verification) runs in the hand-written sm_103a kernels of ``libcutsim.so``
behind the C ABI declared in ``include/cutsim.h``; ``capi`` binds it and
``api`` wraps it with torch-allocated buffers.  Importing this package does
not load the library; the first call does, and fails loudly if it is
missing.
"""

__all__ = ["capi", "api"]


def __getattr__(name):
    if name in ("capi", "api"):
        import importlib

        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
