"""The allocation-free kick (genga_kick_static) against the regular kick.

genga_kick_static exists for callers that cannot allocate device memory (a
framework whose caching allocator already holds the device's free memory, or a
latency-critical loop where cudaMalloc/cudaFree would stall the device); it
keeps its scratch in a fixed device array inside the library.  Here it is
called twice in a row through the C ABI and each result is compared with the
output of genga_kick on a system object, within the kick tolerances used by the
other GPU tests (1e-12 per particle in FP64, 1e-9 mixed).  This file is
collected last so that a stop-at-first-failure run has already run every other
test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from workloads import config_workload, disk

pytestmark = pytest.mark.gpu


def _setup(g, wl, precision):
    import torch
    dev = torch.device("cuda:0")
    pos = torch.tensor(np.ascontiguousarray(wl.x.T), device=dev)
    vel = torch.tensor(np.ascontiguousarray(wl.v.T), device=dev)
    mass = torch.tensor(wl.m, device=dev)
    p = g.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2, f_pc=wl.f_pc,
                         precision=precision)
    s = g.System(pos, vel, mass, p)
    s.rcrit(wl.dt)
    rc = torch.tensor(s.get_rcrit(0), device=dev)
    return s, pos, vel, mass, rc


def _rel(a, b):
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    return (np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)).max()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
@pytest.mark.parametrize("make", [lambda: config_workload(0),
                                  lambda: disk(5003, 0.5, 4.0, 5.0, 91, n_embryos=4)])
def test_kick_static_matches_regular_kick_twice(cuda_lib, precision, tol, make):
    import torch
    g = cuda_lib
    wl = make()
    s, pos, vel, mass, rc = _setup(g, wl, precision)
    n = wl.n
    dt_half = 0.5 * wl.dt
    # reference: the regular kick through a system object
    acc_ref = torch.zeros((3, n), dtype=torch.float64, device="cuda:0")
    s.kick(0.0, precheck=False, acc_out=acc_ref)
    vel_ref = vel.clone()                 # before the kick
    s.kick(dt_half, precheck=False)
    torch.cuda.synchronize()
    vel_kicked = vel.clone()              # after the regular kick
    s.close()

    # first call: accelerations only
    acc1 = torch.full((3, n), np.nan, dtype=torch.float64, device="cuda:0")
    assert g.kick_static(pos, mass, rc, wl.G, 0.0, precision, None, acc1) == 0
    torch.cuda.synchronize()
    assert _rel(acc1, acc_ref) <= tol
    # second call in a row: accelerations and the velocity update
    v2 = vel_ref.clone()
    acc2 = torch.full((3, n), np.nan, dtype=torch.float64, device="cuda:0")
    assert g.kick_static(pos, mass, rc, wl.G, dt_half, precision, v2, acc2) == 0
    torch.cuda.synchronize()
    assert _rel(acc2, acc_ref) <= tol
    dv = (v2 - vel_ref).cpu().numpy()
    dv_ref = (vel_kicked - vel_ref).cpu().numpy()
    assert (np.linalg.norm(dv - dv_ref, axis=0) / np.linalg.norm(dv_ref, axis=0)).max() <= tol


def test_kick_static_rejects_sizes_beyond_its_scratch(cuda_lib):
    import torch
    g = cuda_lib
    n = g.KICK_STATIC_MAX_N + 1
    pos = torch.zeros((3, n), dtype=torch.float64, device="cuda:0")
    mass = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    rc = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    acc = torch.zeros((3, n), dtype=torch.float64, device="cuda:0")
    assert g.kick_static(pos, mass, rc, 1.0, 0.0, 0, None, acc) == -2     # GENGA_ECAPACITY
