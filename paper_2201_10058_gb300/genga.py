"""Thin Python binding of libgenga.so (include/genga.h).

Argument marshalling only: torch CUDA tensors are passed by device pointer,
host arrays by numpy pointer; every step of the integrator runs in the
library's CUDA kernels.  There is no fallback: if the library cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

GENGA_FP64 = 0
GENGA_MIXED = 1
GENGA_GR_IMPLICIT = 1
GENGA_GR_SPLIT = 2
GENGA_KICK_AUTO = 0
GENGA_KICK_TILED = 1
GENGA_KICK_SYMMETRIC = 2
GENGA_BS_PAIRS_AUTO = 0
GENGA_BS_PAIRS_OFF = 1
GENGA_BS_PAIRS_ON = 2

ERRORS = {0: "OK", -1: "EINVAL", -2: "ECAPACITY", -3: "ENONCONV", -4: "ETIMEOUT",
          -5: "EBADSTATE", -6: "ECUDA", -7: "ENOMEM"}

EXPORTED = ["genga_default_params", "genga_create", "genga_destroy", "genga_last_error",
            "genga_set_params", "genga_sync", "genga_rcrit", "genga_set_rcrit", "genga_kick",
            "genga_hc", "genga_drift", "genga_build_encounters", "genga_bs", "genga_step",
            "genga_step_host", "genga_energy", "genga_get_candidates", "genga_get_pairs",
            "genga_get_groups", "genga_get_rcrit", "genga_set_predrift", "genga_get_stats",
            "genga_kick_static", "genga_adjoint_forward", "genga_adjoint_load",
            "genga_adjoint_backward", "genga_adjoint_export", "genga_ensemble_create", "genga_ensemble_destroy",
            "genga_ensemble_last_error", "genga_ensemble_step", "genga_ensemble_set_tile",
            "genga_ensemble_autotune", "genga_ensemble_angmom", "genga_ensemble_get_stats",
            "genga_tune_levels", "genga_set_timing", "genga_get_phase_ms", "genga_phase_name",
            "genga_measure_pipe_rates", "genga_init_system", "genga_step_backward",
            "genga_init_ensemble", "genga_step_ensemble", "genga_set_pair_log",
            "genga_get_pair_log", "genga_set_wait_limits", "genga_set_collisions",
            "genga_get_mergers", "genga_get_alive", "genga_remove_merged", "genga_set_kick_layout",
            "genga_set_bs_pair_mode",
            "genga_get_kick_layout", "genga_measure_fp64_latency"]

NPHASES = 18

KICK_STATIC_MAX_N = 279616


class GengaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("G", C.c_double), ("m_star", C.c_double), ("dt", C.c_double),
                ("n1", C.c_double), ("n2", C.c_double), ("f_pc", C.c_double),
                ("bs_tol", C.c_double), ("slevels", C.c_int32), ("substeps", C.c_int32),
                ("precision", C.c_int32), ("kepler_max_iter", C.c_int32),
                ("bs_max_steps", C.c_int32), ("tp_mode", C.c_int32),
                ("cand_capacity", C.c_int64), ("pair_capacity", C.c_int64),
                ("n_massive", C.c_int64)]


class EnsembleDesc(C.Structure):
    _fields_ = [("n_systems", C.c_int64), ("offsets", C.c_void_p), ("pos", C.c_void_p),
                ("vel", C.c_void_p), ("mass", C.c_void_p), ("spin", C.c_void_p),
                ("radius", C.c_void_p), ("k2", C.c_void_p), ("tau", C.c_void_p),
                ("rg2", C.c_void_p), ("m_star", C.c_void_p), ("dt", C.c_void_p),
                ("star", C.c_void_p), ("c_light", C.c_double), ("gr", C.c_int32),
                ("tides", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("n_candidates", C.c_int64), ("n_pairs", C.c_int64 * 8),
                ("n_groups", C.c_int64), ("max_group", C.c_int64), ("bs_steps", C.c_int64),
                ("bs_rejects", C.c_int64), ("kepler_fail", C.c_int64), ("bs_fail", C.c_int64),
                ("kernel_launches", C.c_int64), ("bs_max_attempts", C.c_int64),
                ("host_syncs", C.c_int64)]

    def as_dict(self) -> dict:
        return {"n_candidates": self.n_candidates, "n_pairs": list(self.n_pairs),
                "n_groups": self.n_groups, "max_group": self.max_group,
                "bs_steps": self.bs_steps, "bs_rejects": self.bs_rejects,
                "kepler_fail": self.kepler_fail, "bs_fail": self.bs_fail,
                "kernel_launches": self.kernel_launches,
                "bs_max_attempts": self.bs_max_attempts, "host_syncs": self.host_syncs}


_lib = None
_lock = threading.Lock()
_VP = C.c_void_p
_P = C.POINTER


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libgenga.so (building it first if needed); raises if it cannot."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing: {path} (run __graft_entry__.build())")
        L = C.CDLL(path)
        sysp = _VP
        L.genga_default_params.argtypes = [_P(Params)]
        L.genga_default_params.restype = None
        L.genga_create.argtypes = [_P(_VP), _P(Params), C.c_int64, _VP, _VP, _VP, _VP]
        L.genga_init_system.argtypes = [_P(_VP), _P(Params), C.c_int64, _VP, _VP, _VP, _VP]
        L.genga_step_backward.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP]
        L.genga_init_ensemble.argtypes = [_P(_VP), _P(Params), _P(EnsembleDesc), _VP]
        L.genga_step_ensemble.argtypes = [_VP, C.c_int64]
        L.genga_destroy.argtypes = [sysp]
        L.genga_destroy.restype = None
        L.genga_last_error.argtypes = [sysp]
        L.genga_last_error.restype = C.c_char_p
        L.genga_set_params.argtypes = [sysp, _P(Params)]
        L.genga_sync.argtypes = [sysp]
        L.genga_rcrit.argtypes = [sysp, C.c_double]
        L.genga_set_rcrit.argtypes = [sysp, _VP]
        L.genga_kick.argtypes = [sysp, C.c_double, C.c_int, _VP]
        L.genga_hc.argtypes = [sysp, C.c_double]
        L.genga_drift.argtypes = [sysp, C.c_double]
        L.genga_build_encounters.argtypes = [sysp, _P(C.c_int64), _P(C.c_int64), _P(C.c_int64)]
        L.genga_bs.argtypes = [sysp, C.c_double]
        L.genga_step.argtypes = [sysp, C.c_int64]
        L.genga_step_host.argtypes = [sysp, _VP, _VP, C.c_int64]
        L.genga_tune_levels.argtypes = [sysp, _VP, _VP, C.c_int32, C.c_int64, _P(C.c_int32), _VP]
        L.genga_energy.argtypes = [sysp, _P(C.c_double), _P(C.c_double)]
        L.genga_get_candidates.argtypes = [sysp, _VP, C.c_int64, _P(C.c_int64)]
        L.genga_get_pairs.argtypes = [sysp, C.c_int, _VP, C.c_int64, _P(C.c_int64)]
        L.genga_get_groups.argtypes = [sysp, _VP]
        L.genga_get_rcrit.argtypes = [sysp, C.c_int, _VP]
        L.genga_set_predrift.argtypes = [sysp, _VP, _VP]
        L.genga_get_stats.argtypes = [sysp, _P(Stats)]
        L.genga_kick_static.argtypes = [C.c_int64, _VP, _VP, _VP, C.c_double, C.c_double, C.c_int,
                                        _VP, _VP, _VP]
        L.genga_adjoint_forward.argtypes = [_VP, C.c_int64, C.c_int64]
        L.genga_adjoint_load.argtypes = [_VP, C.c_int64, C.c_int64, _VP, _VP, _VP]
        L.genga_adjoint_backward.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP]
        L.genga_adjoint_export.argtypes = [_VP, _VP, _VP, _VP, C.c_int64, _P(C.c_int64),
                                           _P(C.c_int64)]
        L.genga_ensemble_create.argtypes = [_P(_VP), _P(Params), _P(EnsembleDesc), _VP]
        L.genga_ensemble_destroy.argtypes = [_VP]
        L.genga_ensemble_destroy.restype = None
        L.genga_ensemble_last_error.argtypes = [_VP]
        L.genga_ensemble_last_error.restype = C.c_char_p
        L.genga_ensemble_step.argtypes = [_VP, C.c_int64]
        L.genga_ensemble_set_tile.argtypes = [_VP, C.c_int, C.c_int]
        L.genga_ensemble_autotune.argtypes = [_VP, C.c_int64, _P(C.c_int), _P(C.c_int)]
        L.genga_ensemble_angmom.argtypes = [_VP, _VP]
        L.genga_ensemble_get_stats.argtypes = [_VP, _P(Stats)]
        L.genga_set_timing.argtypes = [sysp, C.c_int]
        L.genga_get_phase_ms.argtypes = [sysp, _VP, _P(C.c_int64)]
        L.genga_phase_name.argtypes = [C.c_int]
        L.genga_phase_name.restype = C.c_char_p
        L.genga_set_wait_limits.argtypes = [sysp, C.c_double, C.c_double, C.c_int32]
        L.genga_set_collisions.argtypes = [sysp, _VP, _VP, _VP, C.c_double]
        L.genga_get_mergers.argtypes = [sysp, _VP, C.c_int64, _P(C.c_int64), _P(C.c_double)]
        L.genga_get_alive.argtypes = [sysp, _VP]
        L.genga_remove_merged.argtypes = [sysp, _P(C.c_int64), _VP]
        L.genga_set_pair_log.argtypes = [sysp, C.c_int]
        L.genga_set_kick_layout.argtypes = [sysp, C.c_int32, C.c_int32]
        L.genga_set_bs_pair_mode.argtypes = [sysp, C.c_int32]
        L.genga_get_kick_layout.argtypes = [sysp] + [_P(C.c_int32)] * 4
        L.genga_get_pair_log.argtypes = [sysp, _VP, _VP, _VP, C.c_int64, C.c_int64, _P(C.c_int64),
                                         _P(C.c_int64)]
        L.genga_measure_pipe_rates.argtypes = [_P(C.c_double)] * 5
        L.genga_measure_fp64_latency.argtypes = [_P(C.c_double)] * 2
        void_fns = ("genga_default_params", "genga_destroy", "genga_last_error",
                    "genga_ensemble_destroy", "genga_ensemble_last_error", "genga_phase_name")
        for name in EXPORTED:
            if name not in void_fns:
                getattr(L, name).restype = C.c_int
        _lib = L
        return L


def default_params(**kw) -> Params:
    p = Params()
    load().genga_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def kick_static(pos, mass, rc, G: float, dt_half: float, precision: int, vel=None, acc_out=None,
                stream=None) -> int:
    """genga_kick_static on torch CUDA tensors (pos (3,n), mass (n,), rc (n,));
    returns the C status code (0 on success)."""
    import torch
    L = load()
    s = stream if stream is not None else torch.cuda.current_stream()
    ptr = lambda t: None if t is None else _VP(t.data_ptr())
    return L.genga_kick_static(int(mass.shape[0]), ptr(pos), ptr(mass), ptr(rc), G, dt_half,
                               precision, ptr(vel), ptr(acc_out), _VP(s.cuda_stream))


def measure_pipe_rates() -> dict:
    """Thread-level FP64 FMA / add / multiply, FP32 FMA and MUFU rsqrt operations
    per clock per SM on the current device (genga_measure_pipe_rates)."""
    v = [C.c_double() for _ in range(5)]
    rc = load().genga_measure_pipe_rates(*[C.byref(x) for x in v])
    if rc != 0:
        raise GengaError(rc, "genga_measure_pipe_rates failed")
    return dict(zip(("dfma", "dadd", "dmul", "ffma", "rsqrt"), (x.value for x in v)))


def measure_fp64_latency() -> dict:
    """SM cycles per instruction of a dependent FP64 FMA chain, for a full warp
    and for a single thread alone on the device (genga_measure_fp64_latency)."""
    v = [C.c_double() for _ in range(2)]
    rc = load().genga_measure_fp64_latency(*[C.byref(x) for x in v])
    if rc != 0:
        raise GengaError(rc, "genga_measure_fp64_latency failed")
    return {"warp": v[0].value, "lane": v[1].value}


def _np_ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_VP)


class System:
    """One integrated system on the current CUDA device.

    pos, vel: torch float64 CUDA tensors of shape (3, n) (component-major), mass:
    (n,).  The tensors are kept referenced and updated in place.
    """

    def __init__(self, pos, vel, mass, params: Params | None = None, stream=None):
        import torch
        self._lib = load()
        for t, name in ((pos, "pos"), (vel, "vel"), (mass, "mass")):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
        n = mass.shape[0]
        if tuple(pos.shape) != (3, n) or tuple(vel.shape) != (3, n):
            raise ValueError("pos and vel must have shape (3, n)")
        self.pos, self.vel, self.mass = pos, vel, mass
        self.n = int(n)
        self.params = params if params is not None else default_params()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = _VP()
        rc = self._lib.genga_init_system(C.byref(h), C.byref(self.params), self.n, pos.data_ptr(),
                                         vel.data_ptr(), mass.data_ptr(), _VP(self.stream.cuda_stream))
        if rc != 0:
            raise GengaError(rc, "genga_init_system failed")
        self._h = h

    # -- helpers
    def _check(self, rc: int):
        if rc != 0:
            msg = self._lib.genga_last_error(self._h)
            raise GengaError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.genga_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C-ABI calls
    def set_params(self, params: Params):
        self._check(self._lib.genga_set_params(self._h, C.byref(params)))
        self.params = params

    def sync(self):
        self._check(self._lib.genga_sync(self._h))

    def rcrit(self, dt: float):
        self._check(self._lib.genga_rcrit(self._h, dt))

    def set_rcrit(self, rc: np.ndarray):
        rc = np.ascontiguousarray(rc, dtype=np.float64)
        self._check(self._lib.genga_set_rcrit(self._h, _np_ptr(rc)))

    def kick(self, dt_half: float, precheck: bool = False, acc_out=None):
        ptr = None if acc_out is None else _VP(acc_out.data_ptr())
        self._check(self._lib.genga_kick(self._h, dt_half, int(precheck), ptr))

    def hc(self, dt_half: float):
        self._check(self._lib.genga_hc(self._h, dt_half))

    def drift(self, dt: float):
        self._check(self._lib.genga_drift(self._h, dt))

    def build_encounters(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self._lib.genga_build_encounters(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def bs(self, dt: float):
        self._check(self._lib.genga_bs(self._h, dt))

    def step(self, nsteps: int = 1):
        self._check(self._lib.genga_step(self._h, nsteps))

    def tune_levels(self, candidates, trial_steps: int = 2):
        """genga_tune_levels over [(slevels, substeps), ...]; returns the chosen
        index and each candidate's time per step (ms).  The setting becomes the
        system's (self.params follows)."""
        lv = np.ascontiguousarray([c[0] for c in candidates], dtype=np.int32)
        ss = np.ascontiguousarray([c[1] for c in candidates], dtype=np.int32)
        ms = np.zeros(len(candidates), dtype=np.float64)
        best = C.c_int32()
        self._check(self._lib.genga_tune_levels(self._h, _np_ptr(lv), _np_ptr(ss), len(candidates),
                                                trial_steps, C.byref(best), _np_ptr(ms)))
        self.params.slevels, self.params.substeps = (int(v) for v in candidates[best.value])
        return best.value, ms

    def step_host(self, pos_host: np.ndarray, vel_host: np.ndarray, nsteps: int = 1):
        self._check(self._lib.genga_step_host(self._h, _np_ptr(pos_host), _np_ptr(vel_host), nsteps))

    def step_host_ptr(self, pos_ptr: int, vel_ptr: int, nsteps: int = 1):
        self._check(self._lib.genga_step_host(self._h, _VP(pos_ptr), _VP(vel_ptr), nsteps))

    def energy(self):
        E = C.c_double()
        L = (C.c_double * 3)()
        self._check(self._lib.genga_energy(self._h, C.byref(E), L))
        return E.value, np.array(list(L))

    def _pairs(self, fn, *args):
        n = C.c_int64()
        self._check(fn(self._h, *args, None, 0, C.byref(n)))
        out = np.zeros((max(n.value, 1), 2), dtype=np.uint32)
        self._check(fn(self._h, *args, _np_ptr(out), n.value, C.byref(n)))
        return out[:n.value].copy()

    def candidates(self) -> np.ndarray:
        return self._pairs(self._lib.genga_get_candidates)

    def pairs(self, level: int = 0) -> np.ndarray:
        return self._pairs(self._lib.genga_get_pairs, level)

    def groups(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int64)
        self._check(self._lib.genga_get_groups(self._h, _np_ptr(out)))
        return out

    def get_rcrit(self, level: int = 0) -> np.ndarray:
        out = np.zeros(self.n)
        self._check(self._lib.genga_get_rcrit(self._h, level, _np_ptr(out)))
        return out

    def set_predrift(self, pos_soa: np.ndarray, vel_soa: np.ndarray):
        p = np.ascontiguousarray(pos_soa, dtype=np.float64)
        v = np.ascontiguousarray(vel_soa, dtype=np.float64)
        self._check(self._lib.genga_set_predrift(self._h, _np_ptr(p), _np_ptr(v)))

    def stats(self) -> dict:
        st = Stats()
        self._check(self._lib.genga_get_stats(self._h, C.byref(st)))
        return st.as_dict()

    # -- collisions (Sec. 7.1-7.2)
    def set_collisions(self, radius, spin=None, precision: float = 0.0):
        """Switches collisions on.  radius: (n,) float64 CUDA tensor; spin: (3, n)
        (zeros when None).  Mergers then write the masses, radii and spins."""
        import torch
        if spin is None:
            spin = torch.zeros((3, self.n), dtype=torch.float64, device=self.mass.device)
        for t, name, shape in ((radius, "radius", (self.n,)), (spin, "spin", (3, self.n))):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()) or tuple(t.shape) != shape:
                raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of shape {shape}")
        self.radius, self.spin = radius, spin
        self._check(self._lib.genga_set_collisions(self._h, _VP(self.mass.data_ptr()),
                                                   _VP(radius.data_ptr()), _VP(spin.data_ptr()),
                                                   precision))

    def mergers(self):
        """Mergers since the previous call, in integration order: an (k, 6) array
        (time in its Bulirsch-Stoer call, i, j, r_ij, R_i + R_j, dU) and the sum of
        their dU in that order."""
        n, dU = C.c_int64(), C.c_double()
        self._check(self._lib.genga_get_mergers(self._h, None, 0, C.byref(n), None))
        out = np.zeros((max(n.value, 1), 6))
        self._check(self._lib.genga_get_mergers(self._h, _np_ptr(out), n.value, C.byref(n),
                                                C.byref(dU)))
        return out[:n.value].copy(), dU.value

    def alive(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.uint8)
        self._check(self._lib.genga_get_alive(self._h, _np_ptr(out)))
        return out

    def remove_merged(self) -> np.ndarray:
        """Takes the merged-away bodies out (genga_remove_merged); pos, vel, mass,
        radius and spin become views of the compacted bodies.  Returns each new
        body's former index."""
        n_new = C.c_int64()
        idx = np.zeros(self.n, dtype=np.int64)
        self._check(self._lib.genga_remove_merged(self._h, C.byref(n_new), _np_ptr(idx)))
        k = n_new.value
        if k != self.n:
            flat = lambda t, c: t.view(-1)[:c * k]
            self.pos = flat(self.pos, 3).view(3, k)
            self.vel = flat(self.vel, 3).view(3, k)
            self.mass = flat(self.mass, 1)
            self.radius = flat(self.radius, 1)
            self.spin = flat(self.spin, 3).view(3, k)
            self.n = k
        return idx[:k].copy()

    def set_wait_limits(self, bs_group_seconds: float = -1.0, barrier_seconds: float = -1.0,
                        barrier_absent_blocks: int = 0):
        """Wall-clock limits of the bounded device waits (negative: default)."""
        self._check(self._lib.genga_set_wait_limits(self._h, bs_group_seconds, barrier_seconds,
                                                    barrier_absent_blocks))

    def set_kick_layout(self, layout: int = GENGA_KICK_AUTO, P: int = 0):
        """How the all-pairs kick traverses the pairs: GENGA_KICK_AUTO,
        GENGA_KICK_TILED or GENGA_KICK_SYMMETRIC (each unordered pair once),
        with the super-range P (0: chosen for N)."""
        self._check(self._lib.genga_set_kick_layout(self._h, int(layout), int(P)))

    def set_bs_pair_mode(self, mode: int = GENGA_BS_PAIRS_AUTO):
        """Derivative form of the batched Bulirsch-Stoer kernel (groups of more
        than 32 members): GENGA_BS_PAIRS_AUTO, _OFF (member form) or _ON (each
        pair once per column); the results are bit-identical in every mode."""
        self._check(self._lib.genga_set_bs_pair_mode(self._h, int(mode)))

    def kick_layout(self) -> dict:
        """The layout the next kick uses: layout, P, partial slots per body, blocks."""
        v = [C.c_int32() for _ in range(4)]
        self._check(self._lib.genga_get_kick_layout(self._h, *[C.byref(x) for x in v]))
        return {"layout": v[0].value, "P": v[1].value, "slots": v[2].value, "blocks": v[3].value}

    def set_pair_log(self, enable: bool = True):
        """Switches the detection log on or off (and clears it)."""
        self._check(self._lib.genga_set_pair_log(self._h, int(enable)))

    def pair_log(self) -> list:
        """Every detection logged since set_pair_log(True), in order: a list of
        (level, pairs (k, 2) uint32 sorted by (i, j))."""
        ne, npairs = C.c_int64(), C.c_int64()
        self._check(self._lib.genga_get_pair_log(self._h, None, None, None, 0, 0, C.byref(ne),
                                                 C.byref(npairs)))
        lev = np.zeros(max(ne.value, 1), dtype=np.int32)
        off = np.zeros(ne.value + 1, dtype=np.int64)
        ij = np.zeros((max(npairs.value, 1), 2), dtype=np.uint32)
        self._check(self._lib.genga_get_pair_log(self._h, _np_ptr(lev), _np_ptr(off), _np_ptr(ij),
                                                 ne.value, npairs.value, C.byref(ne), C.byref(npairs)))
        return [(int(lev[k]), ij[off[k]:off[k + 1]].copy()) for k in range(ne.value)]

    def set_timing(self, enable: bool = True):
        """Switches the per-phase step timing on or off (clears the sums)."""
        self._check(self._lib.genga_set_timing(self._h, int(enable)))

    def phase_ms(self) -> tuple[dict, int]:
        """Device time per phase summed over the steps timed since set_timing,
        and the number of those steps."""
        out = np.zeros(NPHASES)
        ns = C.c_int64()
        self._check(self._lib.genga_get_phase_ms(self._h, _np_ptr(out), C.byref(ns)))
        names = [self._lib.genga_phase_name(k).decode() for k in range(NPHASES)]
        return dict(zip(names, out.tolist())), ns.value

    # -- adjoint (frozen encounters)
    def adjoint_forward(self, nsteps: int, checkpoint_every: int):
        self._check(self._lib.genga_adjoint_forward(self._h, nsteps, checkpoint_every))

    def adjoint_load(self, checkpoint_every: int, rc_hist: np.ndarray, pairs: list):
        """rc_hist: (nsteps, n) host array; pairs: list of (k_i, 2) uint32 arrays."""
        rc_hist = np.ascontiguousarray(rc_hist, dtype=np.float64)
        nsteps = rc_hist.shape[0]
        offs = np.zeros(nsteps + 1, dtype=np.int64)
        offs[1:] = np.cumsum([len(p) for p in pairs])
        flat = (np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.uint32).reshape(-1, 2)
                                                     for p in pairs]))
                if offs[-1] > 0 else np.zeros((1, 2), dtype=np.uint32))
        self._check(self._lib.genga_adjoint_load(self._h, nsteps, checkpoint_every,
                                                 _np_ptr(rc_hist), _np_ptr(offs), _np_ptr(flat)))

    def adjoint_export(self):
        """Returns (rc_hist (nsteps, n), list of per-step (k, 2) uint32 pair arrays)."""
        ns, npairs = C.c_int64(), C.c_int64()
        self._check(self._lib.genga_adjoint_export(self._h, None, None, None, 0, C.byref(ns),
                                                   C.byref(npairs)))
        rc = np.zeros((ns.value, self.n))
        offs = np.zeros(ns.value + 1, dtype=np.int64)
        flat = np.zeros((max(npairs.value, 1), 2), dtype=np.uint32)
        self._check(self._lib.genga_adjoint_export(self._h, _np_ptr(rc), _np_ptr(offs), _np_ptr(flat),
                                                   npairs.value, C.byref(ns), C.byref(npairs)))
        return rc, [flat[offs[k]:offs[k + 1]].copy() for k in range(ns.value)]

    def adjoint_backward(self, lam_x, lam_v):
        """lam_x, lam_v: (3, n) CUDA tensors; returns (grad_x0, grad_v0, grad_m)."""
        import torch
        gx = torch.empty_like(lam_x)
        gv = torch.empty_like(lam_v)
        gm = torch.empty_like(self.mass)
        self._check(self._lib.genga_step_backward(self._h, _VP(lam_x.data_ptr()),
                                                     _VP(lam_v.data_ptr()), _VP(gx.data_ptr()),
                                                     _VP(gv.data_ptr()), _VP(gm.data_ptr())))
        return gx, gv, gm


class Ensemble:
    """Batched ensemble (include/genga.h, genga_ensemble_*) on torch CUDA tensors.

    `wl` is a workloads.ensemble.Ensemble (numpy); the tensors are copied to the
    device and kept here: pos/vel/spin as (3, n_total), star as (S, 8)."""

    def __init__(self, wl, params: Params | None = None, gr: bool = True, tides: bool = True,
                 stream=None, gr_split: bool = False):
        import torch
        self._lib = load()
        dev = torch.device("cuda", torch.cuda.current_device())
        T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
        self.pos, self.vel, self.spin = T(wl.x.T), T(wl.v.T), T(wl.spin.T)
        self.mass, self.radius, self.k2, self.tau, self.rg2 = (T(wl.m), T(wl.R), T(wl.k2),
                                                                T(wl.tau), T(wl.rg2))
        self.m_star, self.dt, self.star = T(wl.m_star), T(wl.dt), T(wl.star)
        self.offsets = np.ascontiguousarray(wl.offsets, dtype=np.int64)
        p = params if params is not None else default_params(G=wl.G)
        d = EnsembleDesc()
        d.n_systems = wl.n_systems
        d.offsets = self.offsets.ctypes.data
        for name in ("pos", "vel", "mass", "spin", "radius", "k2", "tau", "rg2", "m_star", "dt",
                     "star"):
            setattr(d, name, getattr(self, name).data_ptr())
        d.c_light, d.tides = wl.c_light, int(tides)
        d.gr = (GENGA_GR_SPLIT if gr_split else GENGA_GR_IMPLICIT) if gr else 0
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = _VP()
        rc = self._lib.genga_init_ensemble(C.byref(h), C.byref(p), C.byref(d),
                                           _VP(self.stream.cuda_stream))
        if rc != 0:
            raise GengaError(rc, "genga_init_ensemble failed")
        self._h = h
        self.n_systems = wl.n_systems

    def _check(self, rc):
        if rc != 0:
            msg = self._lib.genga_ensemble_last_error(self._h)
            raise GengaError(rc, msg.decode() if msg else "")

    def step(self, nsteps: int = 1):
        self._check(self._lib.genga_step_ensemble(self._h, nsteps))

    def set_tile(self, threads: int, ctas_per_sm: int):
        self._check(self._lib.genga_ensemble_set_tile(self._h, threads, ctas_per_sm))

    def autotune(self, trial_steps: int = 20):
        t, c = C.c_int(), C.c_int()
        self._check(self._lib.genga_ensemble_autotune(self._h, trial_steps, C.byref(t), C.byref(c)))
        return t.value, c.value

    def angmom(self) -> np.ndarray:
        out = np.zeros((self.n_systems, 3))
        self._check(self._lib.genga_ensemble_angmom(self._h, _np_ptr(out)))
        return out

    def stats(self) -> dict:
        st = Stats()
        self._check(self._lib.genga_ensemble_get_stats(self._h, C.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            self._lib.genga_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
