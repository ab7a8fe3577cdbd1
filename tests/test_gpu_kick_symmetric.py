"""The symmetric kick layout (each unordered pair once, Newton's third law)
against the FP64 CPU oracle, at sizes that span several tiles of 128 and a
ragged last tile, for every super-range P, in both precisions.

The auto layout already takes the symmetric kick at N = 16,384 and above (the
kick tests of test_gpu_parity.py at N = 16,384, 65,540 and 300,000 run it);
here it is forced at small N, where the work items, the diagonal items and the
padding of the last tile are few enough to reach every case:
  * accelerations: per-particle |da|/|a| <= 1e-12 (FP64) / 1e-9 (mixed), and
    the same bound on the difference from the tiled layout;
  * a ring whose neighbours sit inside the changeover band (K < 1 on both
    sides of every neighbour pair);
  * the same result bit for bit on every kick, although the blocks take their
    work items from a counter in whatever order they come;
  * the pre-check fused into the symmetric kick: candidate lists identical to
    the oracle's, including an overflowing list that is regrown;
  * semi-active test particles: kick, candidates and whole steps;
  * whole steps: 10 steps of the N = 2048 disk to 1e-12 (FP64) / 1e-9 (mixed),
    and 100 steps of the encounter-free control.
"""
import numpy as np
import pytest

import oracle as O
from tests import numerics_log
from workloads import G_GAUSS, config_workload, disk, ring

pytestmark = pytest.mark.gpu

G = G_GAUSS
TILE = 128


def _torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def g(cuda_lib):
    return cuda_lib


def _system(g, wl, precision, layout, P=0, **kw):
    torch = _torch()
    dev = torch.device("cuda:0")
    pos = torch.tensor(np.ascontiguousarray(wl.x.T), device=dev)
    vel = torch.tensor(np.ascontiguousarray(wl.v.T), device=dev)
    mass = torch.tensor(wl.m, device=dev)
    p = g.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2, f_pc=wl.f_pc,
                         slevels=wl.slevels, substeps=wl.substeps, precision=precision)
    for k, v in kw.items():
        setattr(p, k, v)
    s = g.System(pos, vel, mass, p)
    s.set_kick_layout(layout, P)
    return s, pos, vel, mass


def _host(t):
    return t.detach().cpu().numpy().T.copy()


def _acc(g, wl, precision, rc, layout, P=0):
    torch = _torch()
    s, *_ = _system(g, wl, precision, layout, P)
    s.set_rcrit(rc)
    acc = torch.zeros((3, wl.n), dtype=torch.float64, device="cuda:0")
    s.kick(0.0, precheck=False, acc_out=acc)
    torch.cuda.synchronize()
    return _host(acc), s


CASES = [(129, 1), (300, 1), (300, 2), (1000, 3), (1000, 6), (3001, 2), (3001, 5)]


@pytest.mark.parametrize("n,P", CASES)
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_symmetric_kick_matches_oracle(g, n, P, precision, tol):
    wl = disk(n, 0.5, 2.0, 2.0, 100 + n, name=f"disk{n}")
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    a, s = _acc(g, wl, precision, rc, g.GENGA_KICK_SYMMETRIC, P)
    lay = s.kick_layout()
    nT = (n + TILE - 1) // TILE
    assert lay["layout"] == g.GENGA_KICK_SYMMETRIC and lay["P"] == P
    assert lay["slots"] == (nT + P - 1) // P
    ref = O.accel(wl.x, wl.m, rc, G, nthreads=8)
    rel = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
    numerics_log.record(f"symmetric kick disk{n} P={P} precision={precision}", "per-particle |da|/|a|",
                        rel.max(), tol)
    assert rel.max() <= tol, (rel.max(), int(np.argmax(rel)))
    at, st = _acc(g, wl, precision, rc, g.GENGA_KICK_TILED)
    assert st.kick_layout()["layout"] == g.GENGA_KICK_TILED
    d = np.linalg.norm(a - at, axis=1) / np.linalg.norm(ref, axis=1)
    assert d.max() <= tol, d.max()
    # momentum balance: the pair forces are equal and opposite up to rounding
    F = wl.m[:, None] * a
    assert np.abs(F.sum(axis=0)).max() < 1e-11 * np.abs(F).sum(axis=0).max()


@pytest.mark.parametrize("n", [1, 2, 3, 33])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_symmetric_kick_tiny_systems(g, n, precision, tol):
    """One ragged tile (one diagonal work item, most of the tile padding): a
    single body feels nothing; two, three and 33 bodies match the oracle."""
    wl = disk(max(n, 2), 0.5, 2.0, 2.0, 40 + n, name=f"disk{n}")
    if n == 1:
        from workloads.disk import Workload
        wl = Workload(name="one", x=wl.x[:1], v=wl.v[:1], m=wl.m[:1], R=wl.R[:1], m_star=wl.m_star, dt=wl.dt,
                      n1=wl.n1, n2=wl.n2, f_pc=wl.f_pc)
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    a, s = _acc(g, wl, precision, rc, g.GENGA_KICK_SYMMETRIC, 1)
    assert s.kick_layout()["slots"] == 1
    if n == 1:
        assert np.all(a == 0.0)
        return
    ref = O.accel(wl.x, wl.m, rc, G, nthreads=1)
    rel = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() <= tol, rel.max()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_symmetric_kick_changeover_band(g, precision, tol):
    """A 300-body ring whose neighbours sit inside the changeover band: the
    rare branch (K from the Newton r, both masses scaled by K) on both sides of
    the pair, inside diagonal and off-diagonal tiles."""
    wl = ring(300)
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    r_nb = np.linalg.norm(wl.x[1:] - wl.x[:-1], axis=1)
    rcij = np.maximum(rc[1:], rc[:-1])
    assert ((r_nb < rcij) & (r_nb > 0.1 * rcij)).sum() > 100     # K strictly between 0 and 1
    for P in (1, 2):
        a, _ = _acc(g, wl, precision, rc, g.GENGA_KICK_SYMMETRIC, P)
        ref = O.accel(wl.x, wl.m, rc, G, nthreads=8)
        rel = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
        numerics_log.record(f"symmetric kick ring300 P={P} precision={precision}", "per-particle |da|/|a|",
                            rel.max(), tol)
        assert rel.max() <= tol, rel.max()


@pytest.mark.parametrize("precision", [0, 1])
def test_symmetric_kick_is_deterministic(g, precision):
    """The persistent blocks take work items in a data-dependent order, but
    every partial sum has one writer and the slots are folded in a fixed
    order: repeated kicks give the same bits."""
    torch = _torch()
    wl = disk(3001, 0.5, 2.0, 2.0, 7, name="disk3001")
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    s, *_ = _system(g, wl, precision, g.GENGA_KICK_SYMMETRIC, 1)
    s.set_rcrit(rc)
    outs = []
    for _ in range(4):
        acc = torch.zeros((3, wl.n), dtype=torch.float64, device="cuda:0")
        s.kick(0.0, precheck=False, acc_out=acc)
        outs.append(acc)
    torch.cuda.synchronize()
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


@pytest.mark.parametrize("n,P", [(300, 1), (1000, 3), (3001, 2)])
@pytest.mark.parametrize("precision", [0, 1])
def test_fused_precheck_candidates_bit_exact(g, n, P, precision):
    """The pre-check rides inside the symmetric kick (float r^2 screen, exact
    FP64 test in the band): the candidate list equals the oracle's, and the
    kick equals the kick without the pre-check."""
    torch = _torch()
    wl = disk(n, 0.9, 1.1, 2.0, 200 + n, name=f"dense{n}")
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    ref = O.precheck(wl.x, rc, wl.f_pc)
    assert len(ref) > 0
    s, pos, vel, mass = _system(g, wl, precision, g.GENGA_KICK_SYMMETRIC, P)
    s.set_rcrit(rc)
    s.kick(0.5 * wl.dt, precheck=True)
    np.testing.assert_array_equal(s.candidates(), ref)
    s2, pos2, vel2, mass2 = _system(g, wl, precision, g.GENGA_KICK_SYMMETRIC, P)
    s2.set_rcrit(rc)
    s2.kick(0.5 * wl.dt, precheck=False)
    torch.cuda.synchronize()
    np.testing.assert_allclose(_host(vel), _host(vel2), rtol=1e-14, atol=0)


def test_fused_precheck_overflow_regrows(g):
    """A candidate list of capacity 16 overflows inside the fused kick; the
    list is regrown and recomputed at the same positions."""
    wl = config_workload(0)
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    torch = _torch()
    dev = torch.device("cuda:0")
    pos = torch.tensor(np.ascontiguousarray(wl.x.T), device=dev)
    vel = torch.tensor(np.ascontiguousarray(wl.v.T), device=dev)
    mass = torch.tensor(wl.m, device=dev)
    p = g.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2, f_pc=wl.f_pc,
                         precision=1, cand_capacity=16)
    s = g.System(pos, vel, mass, p)
    s.set_kick_layout(g.GENGA_KICK_SYMMETRIC, 1)
    s.set_rcrit(rc)
    s.kick(0.5 * wl.dt, precheck=True)
    np.testing.assert_array_equal(s.candidates(), O.precheck(wl.x, rc, wl.f_pc))


@pytest.mark.parametrize("nm,P", [(0, 1), (129, 1), (1500, 1), (1500, 2), (3001, 2)])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_symmetric_kick_test_particles(g, nm, P, precision, tol):
    """Semi-active test particles (Sec. 8.1, bodies from n_massive on) in the
    symmetric layout: work items of test particles only are left out, pairs of
    two test particles are masked in the tiles that straddle n_massive, and a
    test particle folds only the partial sums of the ranges holding large
    bodies."""
    wl = disk(3001, 0.5, 2.0, 2.0, 60, name="disk3001")
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    torch = _torch()
    s, *_ = _system(g, wl, precision, g.GENGA_KICK_SYMMETRIC, P, tp_mode=2, n_massive=nm)
    s.set_rcrit(rc)
    assert s.kick_layout()["layout"] == g.GENGA_KICK_SYMMETRIC
    acc = torch.zeros((3, wl.n), dtype=torch.float64, device="cuda:0")
    s.kick(0.0, precheck=True, acc_out=acc)
    torch.cuda.synchronize()
    a = _host(acc)
    ref = O.accel(wl.x, wl.m, rc, G, nthreads=8, n_massive=nm)
    np.testing.assert_array_equal(s.candidates(), O.precheck(wl.x, rc, wl.f_pc, n_massive=nm))
    if nm == 0:
        assert np.all(a == 0.0)
        return
    rel = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
    numerics_log.record(f"symmetric kick disk3001 test particles from {nm} P={P} precision={precision}",
                        "per-particle |da|/|a|", rel.max(), tol)
    assert rel.max() <= tol, rel.max()


@pytest.mark.parametrize("slevels,substeps", [(1, 1), (2, 10)])
def test_symmetric_test_particle_steps_match_oracle(g, slevels, substeps):
    """5 whole steps of a dense 2048-body disk with test particles from 1500,
    every kick in the symmetric layout, against the oracle (FP64)."""
    wl = disk(2048, 0.5, 1.0, 2.0, 11, name="dense", slevels=slevels, substeps=substeps)
    s, pos, vel, mass = _system(g, wl, 0, g.GENGA_KICK_SYMMETRIC, 2, tp_mode=2, n_massive=1500)
    s.step(5)
    xr, vr, status, ost = O.step(wl.x, wl.v, wl.m, O.make_params(wl, nthreads=8, tp_mode=2, n_massive=1500), 5)
    assert status == 0
    x = _host(pos)
    err = np.linalg.norm(x - xr, axis=1) / np.linalg.norm(xr, axis=1)
    numerics_log.record(f"5 steps dense disk2048 symmetric kick, test particles from 1500, levels=({slevels},{substeps})",
                        "max |dx|/|x|", err.max(), 1e-12)
    assert err.max() <= 1e-12, err.max()


def test_auto_layout_choice(g):
    """AUTO takes the tiled kick at N = 2048 (too few tile pairs to fill the
    GPU) and the symmetric one at N = 16,384; TILED and SYMMETRIC are obeyed."""
    small = config_workload(0)
    s, *_ = _system(g, small, 1, g.GENGA_KICK_AUTO)
    assert s.kick_layout()["layout"] == g.GENGA_KICK_TILED
    big = disk(16384, 0.5, 2.0, 2.0, 3, name="disk16384")
    s, *_ = _system(g, big, 1, g.GENGA_KICK_AUTO)
    lay = s.kick_layout()
    assert lay["layout"] == g.GENGA_KICK_SYMMETRIC and 1 <= lay["P"] <= 6
    s.set_kick_layout(g.GENGA_KICK_TILED)
    assert s.kick_layout()["layout"] == g.GENGA_KICK_TILED
    with pytest.raises(g.GengaError):
        s.set_kick_layout(g.GENGA_KICK_SYMMETRIC, 7)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_symmetric_layout_steps_match_oracle(g, precision, tol):
    """10 whole steps of the N = 2048 disk (encounters, Bulirsch-Stoer groups)
    with every kick in the symmetric layout."""
    wl = config_workload(0)
    s, pos, vel, mass = _system(g, wl, precision, g.GENGA_KICK_SYMMETRIC, 2)
    s.step(10)
    assert s.stats()["n_pairs"][0] > 0
    xr, _, status, _ = O.step(wl.x, wl.v, wl.m, O.make_params(wl, nthreads=8), 10)
    assert status == 0
    x = _host(pos)
    err = np.linalg.norm(x - xr, axis=1) / np.linalg.norm(xr, axis=1)
    numerics_log.record(f"10 steps disk2048 symmetric kick precision={precision}", "max |dx|/|x|",
                        err.max(), tol)
    assert err.max() <= tol, err.max()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_symmetric_layout_encounter_free_control(g, precision, tol):
    """100 steps without encounters (rc = 0, K = 1 for every pair)."""
    wl = config_workload(0)
    wl.n1 = 0.0
    wl.n2 = 0.0
    s, pos, vel, mass = _system(g, wl, precision, g.GENGA_KICK_SYMMETRIC, 1)
    s.step(100)
    xr, *_ = O.step(wl.x, wl.v, wl.m, O.make_params(wl, nthreads=8), 100)
    err = np.linalg.norm(_host(pos) - xr, axis=1) / np.linalg.norm(xr, axis=1)
    assert err.max() <= tol, err.max()
