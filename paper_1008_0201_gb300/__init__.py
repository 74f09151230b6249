"""GB300-native block one-sided Jacobi eigensolver (trigonometric and hyperbolic).

The compute path is the sm_103a library ``_lib/libjacobi_gb300.so`` (C ABI in
``include/jacobi_gb300.h``); ``binding`` is its thin ctypes layer, ``inputs`` the seeded
synthetic workloads.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "binding", "build"]
