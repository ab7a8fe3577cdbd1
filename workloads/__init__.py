"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package holds input generation only (orbital elements to Cartesian
coordinates, unit constants, random draws).  It contains none of the
integrator's arithmetic: no changeover function, kick, drift, detection,
grouping or Bulirsch-Stoer step.
"""
from .disk import (AU_CM, DAY_S, G_GAUSS, K_GAUSS, M_EARTH, MSUN_G, Workload, disk,
                   config_workload, ring)

__all__ = ["AU_CM", "DAY_S", "G_GAUSS", "K_GAUSS", "M_EARTH", "MSUN_G", "Workload",
           "disk", "config_workload", "ring"]
