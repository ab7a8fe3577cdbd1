"""GB300-native hot path of GENGA II's hybrid symplectic integrator.

The compute lives in libgenga.so (CUDA C++ for sm_103a, C ABI in
include/genga.h); ``genga`` is its thin ctypes binding.
"""
from . import genga  # noqa: F401

__all__ = ["genga"]
