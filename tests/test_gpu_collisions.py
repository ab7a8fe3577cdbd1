"""Collisions (Sec. 7.1-7.2, reading R25) on the GPU against the oracle.

The oracle resolves collisions inside its Bulirsch-Stoer group integration
(orc_bs_groups_coll, orc_step_coll) and is pinned by conservation laws, the
survivor rule and a closed-form contact time (tests/test_oracle_collision_pins.py).
Here the CUDA path, through the C ABI, must give the same mergers in the same
order (pairs, survivors), the same alive flags and masses, and states within
the whole-step tolerance of the other parity tests:

* radial two-body infall at collision precision 1e-2 / 1e-4 / 1e-6 and without
  precision (in-block Bulirsch-Stoer, groups of up to 32 members);
* radii too small to touch: the collision instances give the plain result bit
  for bit;
* a dense disk with inflated radii, 8 steps, one level and two levels x 10;
* a 300-body ring whose neighbours overlap at the start: 150 mergers in
  ascending pair order inside one group of 300 (persistent Bulirsch-Stoer);
* removing the merged-away bodies and integrating on, against the oracle run
  on the same compacted bodies.
"""
import numpy as np
import pytest

import oracle as O
from workloads import G_GAUSS, disk, ring

pytestmark = pytest.mark.gpu

G = G_GAUSS


def _t():
    import torch
    return torch


def _system(g, wl, R, S=None, precision=0.0, **kw):
    torch = _t()
    dev = torch.device("cuda:0")
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    pos, vel, mass = T(wl.x.T), T(wl.v.T), T(wl.m)
    p = g.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2, f_pc=wl.f_pc,
                         slevels=wl.slevels, substeps=wl.substeps)
    for k, v in kw.items():
        setattr(p, k, v)
    s = g.System(pos, vel, mass, p)
    S = np.zeros((wl.n, 3)) if S is None else S
    s.set_collisions(T(R), T(S.T), precision)
    return s


def _host(t):
    return t.detach().cpu().numpy().T.copy()


def _same_log(glog, olog, rtol=1e-12, pos_scale=1.0):
    """Same mergers in the same order (pairs exactly); times, radius sums and
    collision energies to rounding; separations to the positions' parity
    (1e-13 of the coordinates: a separation of 2e-4 AU at 0.05 AU carries the
    rounding differences of the coordinates, ~1e-11 of itself)."""
    assert glog.shape == olog.shape, (glog.shape, olog.shape)
    np.testing.assert_array_equal(glog[:, 1:3], olog[:, 1:3])
    np.testing.assert_allclose(glog[:, 0], olog[:, 0], rtol=rtol, atol=1e-300)
    np.testing.assert_allclose(glog[:, 3], olog[:, 3], rtol=0, atol=1e-13 * pos_scale)
    np.testing.assert_allclose(glog[:, 4], olog[:, 4], rtol=rtol, atol=0)
    scale = np.abs(olog[:, 5]).max() if len(olog) else 1.0
    np.testing.assert_allclose(glog[:, 5], olog[:, 5], rtol=0, atol=1e-9 * scale)


def _infall(coll_tol, r0=0.01, Rb=1e-4, mb=1e-3):
    x = np.array([[0.05, 0.0, 0.0], [0.05 + r0, 0.0, 0.0]])
    k = G * 2 * mb
    q = 2 * Rb / r0
    tc = np.sqrt(r0 ** 3 / (2 * k)) * (np.sqrt(q * (1 - q)) + np.arccos(np.sqrt(q)))
    from workloads.disk import Workload
    wl = Workload(name="infall", x=x, v=np.zeros((2, 3)), m=np.array([mb, mb]), R=np.array([Rb, Rb]),
                  m_star=1e-30, dt=1.2 * tc, n1=3.0, n2=0.4, f_pc=4.0)
    return wl


@pytest.mark.parametrize("coll_tol", [1e-2, 1e-4, 1e-6, 0.0])
def test_infall_merger_matches_oracle(cuda_lib, coll_tol):
    g = cuda_lib
    torch = _t()
    wl = _infall(coll_tol)
    rc = np.array([1e9, 1e9])                  # K = 0: the pair is fully in the BS part
    s = _system(g, wl, wl.R, precision=coll_tol)
    s.set_rcrit(rc)
    s.kick(0.0, precheck=True, acc_out=torch.zeros((3, 2), dtype=torch.float64, device="cuda:0"))
    s.set_predrift(wl.x.T, wl.v.T)
    np_, ng_, _ = s.build_encounters()
    assert (np_, ng_) == (1, 1)
    s.bs(wl.dt)
    glog, gdU = s.mergers()
    x, v, m, R, S, alive, U, olog, status, st = O.bs_groups_coll(
        wl.x, wl.v, wl.m, wl.R, np.zeros((2, 3)), rc[None], np.array([[0, 1]], dtype=np.uint32), G,
        wl.m_star, wl.dt, coll_tol=coll_tol)
    assert status == 0 and len(olog) == 1
    _same_log(glog, olog, pos_scale=np.abs(wl.x).max())
    assert gdU == pytest.approx(U, rel=1e-10)
    np.testing.assert_array_equal(s.alive(), alive)
    np.testing.assert_array_equal(s.mass.cpu().numpy(), m)
    np.testing.assert_allclose(s.radius.cpu().numpy(), R, rtol=4e-16, atol=0)
    # the survivor to the state's rounding; the body merged away drifts on from
    # the merger time, which carries the integration's rounding (~1e-12 of it)
    np.testing.assert_allclose(_host(s.pos)[0], x[0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(_host(s.vel)[0], v[0], rtol=0, atol=1e-14 * np.abs(wl.x).max() / wl.dt)
    np.testing.assert_allclose(_host(s.pos)[1], x[1], rtol=1e-11, atol=0)
    if coll_tol > 0:
        t, i, j, r, Rs, dU = glog[0]
        assert 0.0 < (Rs - r) / Rs < coll_tol


def test_no_contact_collision_path_is_bit_identical(cuda_lib):
    """Radii too small to touch: a step through the collision instances of the
    kernels equals the plain step bit for bit."""
    g = cuda_lib
    torch = _t()
    wl = disk(160, 0.9, 1.1, 2.0, 31, name="ring-like")
    s1 = _system(g, wl, np.full(wl.n, 1e-12), precision=1e-3)
    s1.step(2)
    assert s1.stats()["n_groups"] > 0 and len(s1.mergers()[0]) == 0
    dev = torch.device("cuda:0")
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    pos, vel, mass = T(wl.x.T), T(wl.v.T), T(wl.m)
    p = g.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2, f_pc=wl.f_pc)
    s0 = g.System(pos, vel, mass, p)
    s0.step(2)
    assert torch.equal(s1.pos, pos) and torch.equal(s1.vel, vel)


@pytest.mark.parametrize("slevels", [1, 2])
def test_dense_disk_mergers_match_oracle(cuda_lib, slevels):
    """8 steps of a dense disk with inflated radii (R_i + R_j = 6e-3 AU against
    critical radii of ~0.04 AU), collision precision 1e-3."""
    g = cuda_lib
    wl = disk(160, 0.9, 1.1, 2.0, 31, name="ring-like", slevels=slevels, substeps=10)
    R = np.full(wl.n, 3e-3)
    s = _system(g, wl, R, precision=1e-3)
    s.step(8)
    glog, gdU = s.mergers()
    x, v, m, R1, S1, alive, U, olog, status, st = O.step_coll(wl.x, wl.v, wl.m, R, np.zeros((wl.n, 3)),
                                                             O.make_params(wl, nthreads=8), 8,
                                                             coll_tol=1e-3)
    assert status == 0 and len(olog) >= 1
    _same_log(glog, olog)
    assert gdU == pytest.approx(U, rel=1e-12, abs=1e-12 * np.abs(olog[:, 5]).max())
    np.testing.assert_array_equal(s.alive(), alive)
    np.testing.assert_allclose(s.mass.cpu().numpy(), m, rtol=1e-15, atol=0)
    np.testing.assert_allclose(s.radius.cpu().numpy(), R1, rtol=1e-15, atol=0)
    np.testing.assert_allclose(_host(s.spin), S1, rtol=0, atol=1e-12 * np.abs(S1).max())
    xg = _host(s.pos)
    err = np.linalg.norm(xg - x, axis=1) / np.linalg.norm(x, axis=1)
    assert err.max() <= 1e-12, err.max()


def test_giant_group_start_mergers_match_oracle(cuda_lib):
    """A 300-body ring (one close-encounter group of 300: the persistent
    Bulirsch-Stoer kernel) with radii of 0.6 of the neighbour spacing: every
    neighbouring pair overlaps when the group's integration starts, and the
    mergers run in ascending pair order, each seeing those before it -- (0, 1),
    (2, 3), ... -- 150 in all; then the step goes on."""
    g = cuda_lib
    wl = ring(300)
    R = np.full(wl.n, 0.6 * wl.extra["spacing"])
    s = _system(g, wl, R, precision=1e-3)
    s.step(1)
    assert s.stats()["max_group"] == 300
    glog, gdU = s.mergers()
    x, v, m, R1, S1, alive, U, olog, status, st = O.step_coll(wl.x, wl.v, wl.m, R, np.zeros((wl.n, 3)),
                                                             O.make_params(wl, nthreads=8), 1,
                                                             coll_tol=1e-3)
    assert status == 0 and len(olog) == 150
    _same_log(glog, olog)
    np.testing.assert_array_equal(s.alive(), alive)
    np.testing.assert_array_equal(s.mass.cpu().numpy(), m)
    err = np.linalg.norm(_host(s.pos) - x, axis=1) / np.linalg.norm(x, axis=1)
    assert err.max() <= 1e-12, err.max()


def test_remove_merged_then_steps_match_oracle(cuda_lib):
    """After mergers the merged-away bodies are taken out (genga_remove_merged):
    the compacted arrays hold the alive bodies in order, and two more steps
    equal the oracle's on the same compacted bodies."""
    g = cuda_lib
    wl = disk(160, 0.9, 1.1, 2.0, 31, name="ring-like")
    R = np.full(wl.n, 3e-3)
    s = _system(g, wl, R, precision=1e-3)
    s.step(8)
    s.mergers()
    alive = s.alive().astype(bool)
    assert (~alive).sum() >= 1
    before = {k: getattr(s, k).detach().cpu().numpy().copy() for k in ("pos", "vel", "mass", "radius", "spin")}
    old = s.remove_merged()
    k = int(alive.sum())
    assert s.n == k and len(old) == k
    np.testing.assert_array_equal(old, np.nonzero(alive)[0])
    for name in ("pos", "vel", "spin"):
        np.testing.assert_array_equal(getattr(s, name).cpu().numpy(), before[name][:, alive])
    for name in ("mass", "radius"):
        np.testing.assert_array_equal(getattr(s, name).cpu().numpy(), before[name][alive])
    assert s.alive().all()
    xc, vc, mc = before["pos"][:, alive].T.copy(), before["vel"][:, alive].T.copy(), before["mass"][alive]
    Rc, Sc = before["radius"][alive], before["spin"][:, alive].T.copy()
    s.step(2)
    from workloads.disk import Workload
    wc = Workload(name="compacted", x=xc, v=vc, m=mc, R=Rc, m_star=wl.m_star, dt=wl.dt, n1=wl.n1,
                  n2=wl.n2, f_pc=wl.f_pc)
    x, v, m, R1, S1, al, U, olog, status, st = O.step_coll(xc, vc, mc, Rc, Sc, O.make_params(wc, nthreads=8),
                                                          2, coll_tol=1e-3)
    assert status == 0
    _same_log(s.mergers()[0], olog)
    err = np.linalg.norm(_host(s.pos) - x, axis=1) / np.linalg.norm(x, axis=1)
    assert err.max() <= 1e-12, err.max()
