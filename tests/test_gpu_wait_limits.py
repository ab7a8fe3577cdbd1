"""The bounded device waits run out on purpose and the library reports it.

No test here faults or hangs the GPU: each limit is made short (or a barrier
is made to wait for a block that does not exist, a flag nothing sets), the
kernel gives up after the limit, latches the timeout, and returns; the host
reports GENGA_ETIMEOUT with a message, and a new system integrates normally.

* in-block Bulirsch-Stoer (groups of up to 32 members): a 16-body ring forms one
  group; with a zero time limit its integration stops at the first check;
* persistent Bulirsch-Stoer (groups of more than 32): a 300-body ring forms one
  giant group; with one absent block every grid-barrier wait runs out after
  1 ms.
"""
import numpy as np
import pytest

import oracle as O
from workloads import ring

pytestmark = pytest.mark.gpu

ETIMEOUT = -4


def _system(g, wl):
    import torch
    dev = torch.device("cuda:0")
    pos = torch.tensor(np.ascontiguousarray(wl.x.T), device=dev)
    vel = torch.tensor(np.ascontiguousarray(wl.v.T), device=dev)
    mass = torch.tensor(wl.m, device=dev)
    p = g.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2, f_pc=wl.f_pc)
    return g.System(pos, vel, mass, p), pos


def _step_ok_and_matches_oracle(g, wl):
    s, pos = _system(g, wl)
    s.step(1)
    xr, _, st, ost = O.step(wl.x, wl.v, wl.m, O.make_params(wl, nthreads=8), 1)
    assert st == 0 and ost["n_groups"] >= 1
    xg = pos.cpu().numpy().T
    assert np.abs(xg - xr).max() <= 1e-12 * np.abs(xr).max()
    s.close()


def test_in_block_bs_time_limit_reports_timeout(cuda_lib):
    g = cuda_lib
    wl = ring(16)
    s, _ = _system(g, wl)
    s.set_wait_limits(bs_group_seconds=0.0)
    with pytest.raises(g.GengaError) as e:
        s.step(1)
    assert e.value.code == ETIMEOUT
    assert "time limit" in str(e.value)
    s.close()
    _step_ok_and_matches_oracle(g, wl)


def test_grid_barrier_wait_limit_reports_timeout(cuda_lib):
    g = cuda_lib
    wl = ring(300)
    s, _ = _system(g, wl)
    s.set_wait_limits(barrier_seconds=1e-3, barrier_absent_blocks=1)
    with pytest.raises(g.GengaError) as e:
        s.step(1)
    assert e.value.code == ETIMEOUT
    assert "grid-barrier" in str(e.value)
    # the same system, limits back to normal, integrates again
    s.set_wait_limits()
    s.step(1)
    s.close()
    _step_ok_and_matches_oracle(g, wl)


def test_wait_limits_reject_bad_values(cuda_lib):
    g = cuda_lib
    s, _ = _system(g, ring(16))
    with pytest.raises(g.GengaError) as e:
        s.set_wait_limits(barrier_absent_blocks=-1)
    assert e.value.code == -1
    s.close()
