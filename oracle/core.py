"""ctypes binding of the C oracle (numpy in, numpy out).  Test infrastructure."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "genga_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_lib")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OracleParams(C.Structure):
    _fields_ = [("G", C.c_double), ("m_star", C.c_double), ("dt", C.c_double),
                ("n1", C.c_double), ("n2", C.c_double), ("f_pc", C.c_double),
                ("bs_tol", C.c_double), ("slevels", C.c_int32), ("substeps", C.c_int32),
                ("kepler_max_iter", C.c_int32), ("bs_max_steps", C.c_int32),
                ("nthreads", C.c_int32), ("tp_mode", C.c_int32), ("n_massive", C.c_int64)]


class OracleStats(C.Structure):
    _fields_ = [("n_candidates", C.c_int64), ("n_pairs", C.c_int64 * 8),
                ("n_groups", C.c_int64), ("max_group", C.c_int64), ("bs_steps", C.c_int64),
                ("bs_rejects", C.c_int64), ("kepler_fail", C.c_int64), ("bs_fail", C.c_int64),
                ("bs_max_attempts", C.c_int64)]

    def as_dict(self) -> dict:
        return {"n_candidates": self.n_candidates, "n_pairs": list(self.n_pairs),
                "n_groups": self.n_groups, "max_group": self.max_group,
                "bs_steps": self.bs_steps, "bs_rejects": self.bs_rejects,
                "kepler_fail": self.kepler_fail, "bs_fail": self.bs_fail,
                "bs_max_attempts": self.bs_max_attempts}


_D = C.POINTER(C.c_double)
_U32 = C.POINTER(C.c_uint32)
_I64 = C.POINTER(C.c_int64)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_changeover.restype = C.c_double
            L.orc_changeover.argtypes = [C.c_double, C.c_double]
            L.orc_rcrit.argtypes = [C.c_int64, _D, _D, _D, C.c_double, C.c_double, C.c_double,
                                    C.c_double, _D]
            L.orc_accel.argtypes = [C.c_int64, _D, _D, _D, C.c_double, _D, C.c_int]
            L.orc_accel_tp.argtypes = [C.c_int64, C.c_int64, _D, _D, _D, C.c_double, _D, C.c_int]
            L.orc_accel_rows.argtypes = [C.c_int64, _D, _D, _D, C.c_double, _I64, C.c_int64, _D,
                                         C.c_int]
            L.orc_kick.argtypes = [C.c_int64, _D, _D, _D, C.c_double, C.c_double, _D, C.c_int]
            L.orc_pair_log.argtypes = [C.c_int]
            L.orc_pair_log.restype = None
            L.orc_pair_log_size.argtypes = [_I64, _I64, _I64]
            L.orc_pair_log_size.restype = None
            L.orc_pair_log_get.argtypes = [C.POINTER(C.c_int32), _I64, _U32, _I64, _U32]
            L.orc_pair_log_get.restype = None
            L.orc_level_force_parts.argtypes = [C.c_int64, _D, _D, _D, C.c_int, C.c_int64, _U32,
                                                C.c_double, _D, _D, _D]
            L.orc_precheck.restype = C.c_int64
            L.orc_precheck.argtypes = [C.c_int64, _D, _D, C.c_double, _U32, C.c_int64]
            L.orc_precheck_tp.restype = C.c_int64
            L.orc_precheck_tp.argtypes = [C.c_int64, C.c_int64, _D, _D, C.c_double, _U32, C.c_int64]
            L.orc_hc.argtypes = [C.c_int64, _D, _D, _D, C.c_double, C.c_double]
            L.orc_fg.restype = C.c_int64
            L.orc_fg.argtypes = [C.c_int64, _D, _D, C.c_double, C.c_double, C.c_int]
            L.orc_detect.restype = C.c_int64
            L.orc_detect.argtypes = [C.c_int64, _U32, _D, _D, _D, _U32]
            L.orc_group.argtypes = [C.c_int64, C.c_int64, _U32, _I64]
            L.orc_step.restype = C.c_int
            L.orc_step.argtypes = [C.c_int64, _D, _D, _D, C.POINTER(OracleParams), C.c_int64,
                                   C.POINTER(OracleStats)]
            L.orc_bs_groups.restype = C.c_int
            L.orc_bs_groups.argtypes = [C.c_int64, _D, _D, _D, _D, C.c_int, C.c_int64, _U32,
                                        C.c_double, C.c_double, C.c_double, C.c_double, C.c_int,
                                        C.POINTER(OracleStats)]
            L.orc_energy.argtypes = [C.c_int64, _D, _D, _D, C.c_double, C.c_double, _D, _D]
            L.orc_energy_tp.argtypes = [C.c_int64, C.c_int64, _D, _D, _D, C.c_double, C.c_double,
                                        _D, _D]
            L.orc_step_nn.restype = C.c_int
            L.orc_step_nn.argtypes = [C.c_int64, _D, _D, _D, C.POINTER(OracleParams),
                                      C.POINTER(OracleNN), _D, _D, _D, _D, _D, _D, C.c_int64,
                                      C.POINTER(OracleStats)]
            L.orc_angmom_spin.argtypes = [C.c_int64, _D, _D, _D, _D, _D, _D, C.c_double,
                                          C.c_double, C.c_double, _D, _D]
            L.orc_sizeof_nn.restype = C.c_int64
            L.orc_step_record.restype = C.c_int
            L.orc_step_record.argtypes = [C.c_int64, _D, _D, _D, C.POINTER(OracleParams), _D, _U32,
                                          C.c_int64, _I64]
            L.orc_step_frozen.restype = C.c_int
            L.orc_step_frozen.argtypes = [C.c_int64, _D, _D, _D, C.POINTER(OracleParams), _D,
                                          C.c_int64, _U32, _D, _D, _D]
            L.orc_merge.restype = C.c_double
            L.orc_merge.argtypes = [C.c_int64, C.c_int64, _D, _D, _D, _D, _D, C.c_double,
                                    C.POINTER(C.c_int64)]
            _U8 = C.POINTER(C.c_uint8)
            L.orc_bs_groups_coll.restype = C.c_int
            L.orc_bs_groups_coll.argtypes = [C.c_int64, _D, _D, _D, _D, _D, _U8, _D, C.c_int,
                                             C.c_int64, _U32, C.c_double, C.c_double, C.c_double,
                                             C.c_double, C.c_int, C.c_double, _D,
                                             C.POINTER(C.c_int64), _D, C.c_int64,
                                             C.POINTER(OracleStats)]
            L.orc_step_coll.restype = C.c_int
            L.orc_step_coll.argtypes = [C.c_int64, _D, _D, _D, _D, _D, _U8,
                                        C.POINTER(OracleParams), C.c_int64, C.c_double, _D,
                                        C.POINTER(C.c_int64), _D, C.c_int64, C.POINTER(OracleStats)]
            L.orc_sizeof_params.restype = C.c_int64
            L.orc_sizeof_stats.restype = C.c_int64
            assert L.orc_sizeof_params() == C.sizeof(OracleParams)
            assert L.orc_sizeof_stats() == C.sizeof(OracleStats)
            assert L.orc_sizeof_nn() == C.sizeof(OracleNN)
            _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def changeover(r: float, rc: float) -> float:
    return lib().orc_changeover(float(r), float(rc))


def rcrit(x, v, m, m_star, dt, n1=3.0, n2=0.4) -> np.ndarray:
    x, v, m = _f64(x), _f64(v), _f64(m)
    rc = np.empty(m.shape[0])
    lib().orc_rcrit(m.shape[0], _d(x), _d(v), _d(m), m_star, dt, n1, n2, _d(rc))
    return rc


def accel(x, m, rc, G, nthreads: int = 1, n_massive=None) -> np.ndarray:
    """Kick accelerations; with n_massive, bodies i >= n_massive are semi-active
    test particles (no interaction between two of them)."""
    x, m, rc = _f64(x), _f64(m), _f64(rc)
    a = np.empty_like(x)
    n = m.shape[0]
    nm = n if n_massive is None else int(n_massive)
    lib().orc_accel_tp(n, nm, _d(x), _d(m), _d(rc), G, _d(a), nthreads)
    return a


def accel_rows(x, m, rc, G, rows, nthreads: int = 1) -> np.ndarray:
    x, m, rc = _f64(x), _f64(m), _f64(rc)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    a = np.empty((rows.shape[0], 3))
    lib().orc_accel_rows(m.shape[0], _d(x), _d(m), _d(rc), G, rows.ctypes.data_as(_I64),
                         rows.shape[0], _d(a), nthreads)
    return a


def kick(x, v, m, rc, G, dt_half, nthreads: int = 1) -> np.ndarray:
    x, m, rc = _f64(x), _f64(m), _f64(rc)
    v = _f64(v).copy()
    lib().orc_kick(m.shape[0], _d(x), _d(m), _d(rc), G, dt_half, _d(v), nthreads)
    return v


def pair_log(enable: bool):
    """Switches the oracle's detection log on or off (and clears it)."""
    lib().orc_pair_log(int(enable))


def pair_log_get():
    """The detections logged since pair_log(True), in order: a list of
    (level, pairs (k, 2) uint32 in output order, borderline candidates (b, 2))."""
    L = lib()
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    L.orc_pair_log_size(C.byref(a), C.byref(b), C.byref(c))
    nev, npairs, nb = a.value, b.value, c.value
    lev = np.zeros(max(nev, 1), dtype=np.int32)
    off = np.zeros(nev + 1, dtype=np.int64)
    boff = np.zeros(nev + 1, dtype=np.int64)
    pairs = np.zeros((max(npairs, 1), 2), dtype=np.uint32)
    border = np.zeros((max(nb, 1), 2), dtype=np.uint32)
    L.orc_pair_log_get(lev.ctypes.data_as(C.POINTER(C.c_int32)), off.ctypes.data_as(_I64),
                       pairs.ctypes.data_as(_U32), boff.ctypes.data_as(_I64), border.ctypes.data_as(_U32))
    return [(int(lev[k]), pairs[off[k]:off[k + 1]].copy(), border[boff[k]:boff[k + 1]].copy())
            for k in range(nev)]


def level_force_parts(x, m, rc_levels, pairs, G):
    """The oracle's level split of the pair accelerations (test hook): returns
    (kick (n,3), kickS (nlev-1, n, 3), bs (n,3)) for the ascending pair list
    `pairs` (k, 2) used at every level; rc_levels (nlev, n)."""
    x = _f64(x)
    m = _f64(m)
    rc_levels = _f64(rc_levels)
    nlev, n = rc_levels.shape
    pairs = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
    pp = pairs if len(pairs) else np.zeros((1, 2), dtype=np.uint32)
    ak = np.zeros((n, 3))
    aks = np.zeros((max(nlev - 1, 1), n, 3))
    ab = np.zeros((n, 3))
    rc = lib().orc_level_force_parts(n, _d(x), _d(m), _d(rc_levels), nlev, len(pairs),
                                     pp.ctypes.data_as(_U32), G, _d(ak), _d(aks), _d(ab))
    if rc != 0:
        raise ValueError("orc_level_force_parts: bad pair list or level count")
    return ak, aks[:nlev - 1], ab


def precheck(x, rc, f_pc, n_massive=None) -> np.ndarray:
    x, rc = _f64(x), _f64(rc)
    n = rc.shape[0]
    nm = n if n_massive is None else int(n_massive)
    cap = 4096
    while True:
        out = np.empty((cap, 2), dtype=np.uint32)
        c = lib().orc_precheck_tp(n, nm, _d(x), _d(rc), f_pc, out.ctypes.data_as(_U32), cap)
        if c <= cap:
            return out[:c].copy()
        cap = int(c)


def hc(x, v, m, m_star, dt_half) -> np.ndarray:
    x = _f64(x).copy()
    v, m = _f64(v), _f64(m)
    lib().orc_hc(m.shape[0], _d(x), _d(v), _d(m), m_star, dt_half)
    return x


def drift(x, v, mu, dt, max_iter: int = 50):
    """Kepler drift of every body; returns (x, v, number of non-converged)."""
    x, v = _f64(x).copy(), _f64(v).copy()
    fails = lib().orc_fg(x.shape[0], _d(x), _d(v), mu, dt, max_iter)
    return x, v, int(fails)


def detect(cand, xpre, xpost, rc) -> np.ndarray:
    cand = np.ascontiguousarray(cand, dtype=np.uint32).reshape(-1, 2)
    xpre, xpost, rc = _f64(xpre), _f64(xpost), _f64(rc)
    out = np.empty((max(cand.shape[0], 1), 2), dtype=np.uint32)
    c = lib().orc_detect(cand.shape[0], cand.ctypes.data_as(_U32), _d(xpre), _d(xpost), _d(rc),
                         out.ctypes.data_as(_U32))
    return out[:c].copy()


def group(n, pairs) -> np.ndarray:
    pairs = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
    label = np.empty(n, dtype=np.int64)
    lib().orc_group(n, pairs.shape[0], pairs.ctypes.data_as(_U32), label.ctypes.data_as(_I64))
    return label


def make_params(wl=None, **kw) -> OracleParams:
    p = OracleParams()
    defaults = dict(G=0.01720209895 ** 2, m_star=1.0, dt=6.0875, n1=3.0, n2=0.4, f_pc=4.0,
                    bs_tol=1e-13, slevels=1, substeps=1, kepler_max_iter=50,
                    bs_max_steps=100000, nthreads=1, tp_mode=0, n_massive=0)
    if wl is not None:
        for k in ("G", "m_star", "dt", "n1", "n2", "f_pc", "slevels", "substeps"):
            defaults[k] = getattr(wl, k)
    defaults.update(kw)
    for k, val in defaults.items():
        setattr(p, k, val)
    return p


def step(x, v, m, params: OracleParams, nsteps: int = 1):
    """Advance nsteps; returns (x, v, status, stats dict)."""
    x, v, m = _f64(x).copy(), _f64(v).copy(), _f64(m)
    st = OracleStats()
    status = lib().orc_step(m.shape[0], _d(x), _d(v), _d(m), C.byref(params), nsteps,
                            C.byref(st))
    return x, v, int(status), st.as_dict()


def bs_groups(x, v, m, rc_levels, pairs, G, m_star, dt, tol=1e-13, max_steps=100000):
    """BS-integrate every group of the ascending pair list over dt.

    rc_levels is (nlev, n); returns (x, v, status, stats dict)."""
    x, v, m = _f64(x).copy(), _f64(v).copy(), _f64(m)
    rcl = _f64(np.atleast_2d(rc_levels))
    pairs = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
    st = OracleStats()
    status = lib().orc_bs_groups(m.shape[0], _d(x), _d(v), _d(m), _d(rcl), rcl.shape[0],
                                 pairs.shape[0], pairs.ctypes.data_as(_U32), G, m_star, dt, tol,
                                 max_steps, C.byref(st))
    return x, v, int(status), st.as_dict()


class OracleNN(C.Structure):
    _fields_ = [("gr", C.c_int32), ("tides", C.c_int32), ("implicit_max_iter", C.c_int32),
                ("gr_split", C.c_int32), ("c_light", C.c_double), ("R_star", C.c_double),
                ("k2_star", C.c_double), ("tau_star", C.c_double), ("rg2_star", C.c_double)]


def make_nn(gr=True, tides=True, c_light=173.1446326846693, R_star=0.0, k2_star=0.0,
            tau_star=0.0, rg2_star=0.0, implicit_max_iter=10, gr_split=False) -> OracleNN:
    """GR by Eq. apn with the implicit midpoint rule, or with gr_split by the
    Hamiltonian splitting of Sec. 3.1 (reading R28)."""
    nn = OracleNN()
    nn.gr, nn.tides, nn.implicit_max_iter = int(gr), int(tides), implicit_max_iter
    nn.gr_split = int(gr_split)
    nn.c_light, nn.R_star, nn.k2_star, nn.tau_star, nn.rg2_star = (c_light, R_star, k2_star,
                                                                   tau_star, rg2_star)
    return nn


def step_nn(x, v, m, params: OracleParams, nn: OracleNN, R, k2, tau, rg2, spin, spin_star,
            nsteps: int = 1):
    """Steps with GR/tides; returns (x, v, spin, spin_star, status, stats)."""
    x, v, m = _f64(x).copy(), _f64(v).copy(), _f64(m)
    R, k2, tau, rg2 = _f64(R), _f64(k2), _f64(tau), _f64(rg2)
    spin, spin_star = _f64(spin).copy(), _f64(spin_star).copy()
    st = OracleStats()
    status = lib().orc_step_nn(m.shape[0], _d(x), _d(v), _d(m), C.byref(params), C.byref(nn),
                               _d(R), _d(k2), _d(tau), _d(rg2), _d(spin), _d(spin_star), nsteps,
                               C.byref(st))
    return x, v, spin, spin_star, int(status), st.as_dict()


def angmom_spin(x, v, m, R, rg2, spin, m_star, R_star, rg2_star, spin_star):
    L = np.zeros(3)
    args = [_f64(a) for a in (x, v, m, R, rg2, spin)]
    lib().orc_angmom_spin(m.shape[0], *[_d(a) for a in args], m_star, R_star, rg2_star,
                          _d(_f64(spin_star)), _d(L))
    return L


def step_record(x, v, m, params: OracleParams):
    """One step (original scheme); returns (x, v, rc, pairs, status)."""
    x, v, m = _f64(x).copy(), _f64(v).copy(), _f64(m)
    n = m.shape[0]
    rc = np.zeros(n)
    cap = 4096
    while True:
        xx, vv = x.copy(), v.copy()
        pairs = np.zeros((cap, 2), dtype=np.uint32)
        npairs = C.c_int64()
        st = lib().orc_step_record(n, _d(xx), _d(vv), _d(m), C.byref(params), _d(rc),
                                   pairs.ctypes.data_as(_U32), cap, C.byref(npairs))
        if npairs.value <= cap:
            return xx, vv, rc, pairs[:npairs.value].copy(), int(st)
        cap = npairs.value


def step_frozen(x, v, m, params: OracleParams, rc, pairs, dx=None, dv=None, dm=None):
    """One step with frozen rc/pairs; with tangents when dx is given.
    Returns (x, v, dx, dv, status)."""
    x, v, m, rc = _f64(x).copy(), _f64(v).copy(), _f64(m), _f64(rc)
    pairs = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
    if dx is not None:
        dx, dv, dm = _f64(dx).copy(), _f64(dv).copy(), _f64(dm)
        st = lib().orc_step_frozen(m.shape[0], _d(x), _d(v), _d(m), C.byref(params), _d(rc),
                                   pairs.shape[0], pairs.ctypes.data_as(_U32), _d(dx), _d(dv),
                                   _d(dm))
    else:
        st = lib().orc_step_frozen(m.shape[0], _d(x), _d(v), _d(m), C.byref(params), _d(rc),
                                   pairs.shape[0], pairs.ctypes.data_as(_U32), None, None, None)
    return x, v, dx, dv, int(st)


def energy(x, v, m, m_star, G, n_massive=None):
    x, v, m = _f64(x), _f64(v), _f64(m)
    E = np.zeros(1)
    L = np.zeros(3)
    n = m.shape[0]
    nm = n if n_massive is None else int(n_massive)
    lib().orc_energy_tp(n, nm, _d(x), _d(v), _d(m), m_star, G, _d(E), _d(L))
    return float(E[0]), L


# ---------------------------------------------------------------- collisions (Sec. 7.1-7.2)
def merge(i, j, x, v, m, R, S, G):
    """Sec. 7.1 merger of bodies i and j (copies of the arrays are changed and
    returned): (x, v, m, R, S, dU, survivor)."""
    x, v, m, R, S = (_f64(a).copy() for a in (x, v, m, R, S))
    sv = C.c_int64()
    dU = lib().orc_merge(int(i), int(j), _d(x), _d(v), _d(m), _d(R), _d(S), G, C.byref(sv))
    return x, v, m, R, S, float(dU), int(sv.value)


def _coll_state(x, v, m, R, S, alive):
    x, v, m, R, S = (_f64(a).copy() for a in (x, v, m, R, S))
    n = m.shape[0]
    alive = np.ones(n, dtype=np.uint8) if alive is None else np.ascontiguousarray(alive, dtype=np.uint8).copy()
    return x, v, m, R, S, alive


def bs_groups_coll(x, v, m, R, S, rc_levels, pairs, G, m_star, dt, tol=1e-13, max_steps=100000,
                   coll_tol=0.0, alive=None):
    """BS of every group with collisions (R25).  Returns (x, v, m, R, S, alive,
    U, log, status, stats); log has one row per merger: time in the call, i, j,
    r_ij, R_i + R_j, Delta U."""
    x, v, m, R, S, alive = _coll_state(x, v, m, R, S, alive)
    rcl = _f64(np.atleast_2d(rc_levels))
    pairs = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
    U = np.zeros(1)
    nc = C.c_int64(0)
    log = np.zeros((max(m.shape[0], 1), 6))
    st = OracleStats()
    status = lib().orc_bs_groups_coll(m.shape[0], _d(x), _d(v), _d(m), _d(R), _d(S),
                                      alive.ctypes.data_as(C.POINTER(C.c_uint8)), _d(rcl),
                                      rcl.shape[0], pairs.shape[0], pairs.ctypes.data_as(_U32),
                                      G, m_star, dt, tol, max_steps, coll_tol, _d(U), C.byref(nc),
                                      _d(log), log.shape[0], C.byref(st))
    return (x, v, m, R, S, alive, float(U[0]), log[:nc.value].copy(), int(status), st.as_dict())


def step_coll(x, v, m, R, S, params: OracleParams, nsteps: int = 1, coll_tol=0.0, alive=None):
    """Steps with collisions (R25).  Returns (x, v, m, R, S, alive, U, log,
    status, stats) as bs_groups_coll (log times from the start of each BS call)."""
    x, v, m, R, S, alive = _coll_state(x, v, m, R, S, alive)
    U = np.zeros(1)
    nc = C.c_int64(0)
    log = np.zeros((max(m.shape[0], 1), 6))
    st = OracleStats()
    status = lib().orc_step_coll(m.shape[0], _d(x), _d(v), _d(m), _d(R), _d(S),
                                 alive.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(params),
                                 nsteps, coll_tol, _d(U), C.byref(nc), _d(log), log.shape[0],
                                 C.byref(st))
    return (x, v, m, R, S, alive, float(U[0]), log[:nc.value].copy(), int(status), st.as_dict())

