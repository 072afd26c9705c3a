"""GB300-native azimuthal integration with pixel splitting.

Implements the method of Kieffer & Ashiotis, "PyFAI: a Python library for high performance
azimuthal integration on GPU" (EuroSciPy 2014) as a C ABI over hand-written sm_103a CUDA
kernels (include/azint.h).  This package is the Python binding; importing it does not load
the CUDA library until the first call.
"""
from __future__ import annotations

__all__ = ["Geometry", "Integrator", "MultiPlan", "AzimuthalIntegrate", "integrate", "build",
           "AzError"]


def build(force: bool = False) -> str:
    """Compile libazint.so for sm_103a (in-tree) and return its path."""
    from . import _build
    return _build.build(force=force)


def __getattr__(name):
    if name in ("Geometry", "Integrator", "MultiPlan", "AzError"):
        from . import api
        return getattr(api, name)
    if name in ("AzimuthalIntegrate", "integrate"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
