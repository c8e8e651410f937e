"""GB300 spherical centroidal Voronoi tessellation engine (Lloyd-preconditioned LBFGS).

The computation lives in the CUDA library ``libscvt.so`` behind the C ABI of
``include/scvt.h``; ``capi`` binds it one to one and ``Engine`` wraps it for
PyTorch tensors.  ``inputs`` generates seeded synthetic workloads.
"""
__all__ = ["capi", "engine", "inputs", "build", "Engine"]


def __getattr__(name):
    if name == "Engine":
        from .engine import Engine
        return Engine
    raise AttributeError(name)
