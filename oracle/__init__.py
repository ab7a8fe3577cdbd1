"""FP64 CPU oracle of the GENGA II hybrid symplectic step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline and
reference legs may import this package.  It is a plain C implementation
(``genga_oracle.c``) loaded through ctypes; it shares no code with the CUDA
library.  See ``genga_oracle.c`` for the readings taken where the paper is
silent.
"""
from .core import (OracleNN, OracleParams, OracleStats, accel, accel_rows, angmom_spin, bs_groups,
                   bs_groups_coll, build, changeover, detect, drift, energy, group, hc, kick,
                   level_force_parts, lib, make_nn, make_params, merge, pair_log, pair_log_get,
                   precheck, rcrit, step, step_coll, step_frozen, step_nn, step_record)

__all__ = ["OracleNN", "OracleParams", "OracleStats", "accel", "accel_rows", "angmom_spin",
           "bs_groups", "bs_groups_coll", "build", "changeover", "detect", "drift", "energy",
           "group", "hc", "kick", "level_force_parts", "lib", "make_nn", "make_params", "merge",
           "pair_log", "pair_log_get", "precheck", "rcrit", "step", "step_coll", "step_frozen",
           "step_nn", "step_record"]
