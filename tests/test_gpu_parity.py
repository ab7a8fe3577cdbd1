"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every input is seeded and synthetic; every expected value comes from the
oracle on the same inputs.  Tolerances:
  * integer/index results (candidates, encounter pairs, group labels): exact;
  * FP64 kick: per-particle |da|/|a| <= 1e-12;
  * mixed kick: per-particle |da|/|a| <= 1e-9 (the target stated for the mixed form);
  * drift, HC, BS, energy: a few ulp to 1e-12 relative (see each test);
  * whole steps: max relative position error <= 1e-12 after 10 steps at N = 2048 and
    in the encounter-free control after 100 steps; with encounters, 100 steps agree
    to within 3x the oracle's own spread under a one-ulp input perturbation.
"""
import os

import numpy as np
import pytest

import oracle as O
from tests import borderline, numerics_log
from workloads import G_GAUSS, config_workload, disk, ring

pytestmark = pytest.mark.gpu

G = G_GAUSS


def _torch():
    import torch
    return torch


def _system(g, wl, precision=0, **kw):
    torch = _torch()
    dev = torch.device("cuda:0")
    pos = torch.tensor(np.ascontiguousarray(wl.x.T), device=dev)
    vel = torch.tensor(np.ascontiguousarray(wl.v.T), device=dev)
    mass = torch.tensor(wl.m, device=dev)
    p = g.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2, f_pc=wl.f_pc,
                         slevels=wl.slevels, substeps=wl.substeps, precision=precision)
    for k, v in kw.items():
        setattr(p, k, v)
    return g.System(pos, vel, mass, p), pos, vel, mass


def _host(t):
    return t.detach().cpu().numpy().T.copy()


@pytest.fixture(scope="module")
def g(cuda_lib):
    return cuda_lib


SIZES = [("disk2048", lambda: config_workload(0)),
         ("disk3001_ragged", lambda: disk(3001, 0.5, 2.0, 2.0, 77, name="ragged"))]


# ---------------------------------------------------------------- Eq. rcrit
@pytest.mark.parametrize("name,make", SIZES)
def test_rcrit_matches_oracle(g, name, make):
    wl = make()
    s, *_ = _system(g, wl)
    s.rcrit(wl.dt)
    rc = s.get_rcrit(0)
    ref = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    np.testing.assert_allclose(rc, ref, rtol=4e-16, atol=0)


# ---------------------------------------------------------------- Eq. Hb kick
def _acc(g, wl, precision, rc):
    torch = _torch()
    s, pos, vel, mass = _system(g, wl, precision)
    s.set_rcrit(rc)
    acc = torch.zeros((3, wl.n), dtype=torch.float64, device="cuda:0")
    s.kick(0.0, precheck=False, acc_out=acc)
    torch.cuda.synchronize()
    return _host(acc)


def _abs_sum(wl, rc, rows):
    """sum_j |a_ij| = sum_j G m_j K(r_ij / rc_ij) / r_ij^2 for the given rows, the
    normalisation for near-cancelling sums (K as the kick uses it: y = (r/rc -
    0.1)/0.9 clamped to [0, 1], K = y^2 / (2y^2 - 2y + 1))."""
    out = []
    for i in rows:
        d = wl.x - wl.x[i]
        r = np.linalg.norm(d, axis=1)
        r[i] = np.inf
        y = np.clip((r / np.maximum(rc, rc[i]) - 0.1) / 0.9, 0.0, 1.0)
        K = y * y / (2 * y * y - 2 * y + 1)
        out.append(G * (wl.m * K / r ** 2).sum())
    return np.array(out)


@pytest.mark.parametrize("name,make", SIZES)
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_kick_acceleration_matches_oracle(g, name, make, precision, tol):
    wl = make()
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    a = _acc(g, wl, precision, rc)
    ref = O.accel(wl.x, wl.m, rc, G, nthreads=8)
    rel = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
    numerics_log.record(f"kick {name} precision={precision}", "per-particle |da|/|a|", rel.max(), tol)
    # the same error normalised by sum_j |a_ij| (insensitive to near-cancelling sums)
    rows = np.arange(wl.n)
    reln = np.linalg.norm(a - ref, axis=1) / _abs_sum(wl, rc, rows)
    numerics_log.record(f"kick {name} precision={precision}", "per-particle |da|/sum_j|a_ij|",
                        reln.max(), tol)
    assert rel.max() <= tol, (rel.max(), np.argmax(rel))
    assert reln.max() <= tol
    # momentum balance of the GPU kick (force scaling is symmetric)
    F = wl.m[:, None] * a
    assert np.abs(F.sum(axis=0)).max() < 1e-11 * np.abs(F).sum(axis=0).max()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_kick_config1_size(g, precision, tol):
    """N = 16384 disk (the FP64-vs-mixed kick configuration): every particle."""
    wl = config_workload(1)
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    a = _acc(g, wl, precision, rc)
    ref = O.accel(wl.x, wl.m, rc, G, nthreads=16)
    rel = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
    numerics_log.record(f"kick disk16384 precision={precision}", "per-particle |da|/|a|", rel.max(), tol)
    assert rel.max() <= tol


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_kick_bench_size_sampled_rows(g, precision, tol):
    """The bench disk (N = 65,540, launch configuration of bench.py): 512 sampled
    rows against the oracle computed row by row; candidates checked for those rows."""
    wl = config_workload(2)
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    a = _acc(g, wl, precision, rc)
    rows = np.random.default_rng(5).choice(wl.n, 512, replace=False)
    rows = np.concatenate([rows, [0, wl.n - 1, wl.n - 2, wl.n - 4]])   # embryos and the tail
    ref = O.accel_rows(wl.x, wl.m, rc, G, rows, nthreads=16)
    rel = np.linalg.norm(a[rows] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    numerics_log.record(f"kick disk65540 (516 rows) precision={precision}", "per-particle |da|/|a|",
                        rel.max(), tol)
    assert rel.max() <= tol, rel.max()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_kick_large_n_sampled_rows(g, precision, tol):
    """N = 300,000 (more source chunks than the partial-sum cap allows at 16 tiles
    each, so the chunks widen): 64 sampled rows, the first and the last, against
    the oracle row by row."""
    wl = disk(300000, 0.5, 4.0, 5.0, 91, name="disk300k")
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    a = _acc(g, wl, precision, rc)
    rows = np.concatenate([np.random.default_rng(9).choice(wl.n, 62, replace=False), [0, wl.n - 1]])
    ref = O.accel_rows(wl.x, wl.m, rc, G, rows, nthreads=16)
    rel = np.linalg.norm(a[rows] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    numerics_log.record(f"kick disk300000 (64 rows) precision={precision}", "per-particle |da|/|a|",
                        rel.max(), tol)
    assert rel.max() <= tol, rel.max()


def test_kick_applies_velocity_update(g):
    wl = config_workload(0)
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    s, pos, vel, mass = _system(g, wl, 0)
    s.set_rcrit(rc)
    s.kick(0.5 * wl.dt, precheck=False)
    ref = O.kick(wl.x, wl.v, wl.m, rc, G, 0.5 * wl.dt, nthreads=8)
    np.testing.assert_allclose(_host(vel), ref, rtol=0, atol=1e-17)


@pytest.mark.parametrize("name,make", SIZES + [("ring64", lambda: ring(64))])
def test_precheck_candidates_bit_exact(g, name, make):
    wl = make()
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    s, *_ = _system(g, wl, 1)
    s.set_rcrit(rc)
    s.kick(0.5 * wl.dt, precheck=True)
    cand = s.candidates()
    ref = O.precheck(wl.x, rc, wl.f_pc)
    assert len(ref) > 0
    np.testing.assert_array_equal(cand, ref)


def test_candidate_list_grows_on_overflow(g):
    wl = config_workload(0)
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    s, *_ = _system(g, wl, 1, cand_capacity=16)
    s.set_rcrit(rc)
    s.kick(0.5 * wl.dt, precheck=True)
    np.testing.assert_array_equal(s.candidates(), O.precheck(wl.x, rc, wl.f_pc))


def test_step_candidate_overflow_uses_step_start_positions(g):
    """Inside a whole step the overflowed list is recomputed before HC and the
    drift move the bodies: candidates, pairs and positions as without overflow."""
    wl = config_workload(0)
    s, pos, vel, mass = _system(g, wl, 0, cand_capacity=16)
    s.step(1)
    st = s.stats()
    xr, vr, status, ost = O.step(wl.x, wl.v, wl.m, O.make_params(wl, nthreads=8), 1)
    assert status == 0 and ost["n_candidates"] > 16
    assert st["n_candidates"] == ost["n_candidates"]
    assert st["n_pairs"][0] == ost["n_pairs"][0]
    err = _rel_pos_err(_host(pos), xr)
    assert err.max() <= 1e-12, err.max()


# ---------------------------------------------------------------- Eq. Hc and Eq. Ha Kepler drift
def test_hc_matches_oracle(g):
    wl = config_workload(0)
    s, pos, vel, mass = _system(g, wl)
    s.hc(0.5 * wl.dt)
    ref = O.hc(wl.x, wl.v, wl.m, wl.m_star, 0.5 * wl.dt)
    np.testing.assert_allclose(_host(pos), ref, rtol=0, atol=4e-16 * np.abs(wl.x).max())


@pytest.mark.parametrize("dt", [6.0875, 0.5, 60.0, -6.0875])
def test_drift_matches_oracle(g, dt):
    wl = config_workload(0)
    s, pos, vel, mass = _system(g, wl)
    s.drift(dt)
    xr, vr, fails = O.drift(wl.x, wl.v, G * wl.m_star, dt)
    assert fails == 0
    # the universal-variable solve's rounding grows with the anomaly swept (|dt|)
    scale = max(1.0, abs(dt) / 6.0875)
    np.testing.assert_allclose(_host(pos), xr, rtol=0, atol=5e-15 * scale * np.abs(xr).max())
    np.testing.assert_allclose(_host(vel), vr, rtol=0, atol=5e-15 * scale * np.abs(vr).max())


# ---------------------------------------------------------------- detection, grouping, BS
def _encounter_setup(g, wl):
    """Oracle states for one step's detection: pre-drift (after Kick + HC) and post-drift."""
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    v1 = O.kick(wl.x, wl.v, wl.m, rc, G, 0.5 * wl.dt, nthreads=8)
    x1 = O.hc(wl.x, v1, wl.m, wl.m_star, 0.5 * wl.dt)
    x2, v2, _ = O.drift(x1, v1, G * wl.m_star, wl.dt)
    cand = O.precheck(wl.x, rc, wl.f_pc)
    return rc, x1, v1, x2, v2, cand


@pytest.mark.parametrize("name,make", SIZES)
def test_detection_and_grouping_bit_exact(g, name, make):
    torch = _torch()
    wl = make()
    rc, x1, v1, x2, v2, cand = _encounter_setup(g, wl)
    s, pos, vel, mass = _system(g, wl, 0)
    s.set_rcrit(rc)
    s.kick(0.0, precheck=True, acc_out=torch.zeros((3, wl.n), dtype=torch.float64, device="cuda:0"))
    s.set_predrift(x1.T, v1.T)
    pos.copy_(torch.tensor(x2.T.copy()))
    vel.copy_(torch.tensor(v2.T.copy()))
    npairs, ngroups, maxg = s.build_encounters()
    ref_pairs = O.detect(cand, x1, x2, rc)
    borderline.record(name, cand, x1, x2, rc)
    assert npairs == len(ref_pairs) > 0
    np.testing.assert_array_equal(s.pairs(0), ref_pairs)
    lab = s.groups()
    ref_lab = O.group(wl.n, ref_pairs)
    np.testing.assert_array_equal(lab, ref_lab)
    assert ngroups == len(np.unique(ref_lab[ref_lab >= 0]))
    assert maxg == np.bincount(ref_lab[ref_lab >= 0]).max()


def test_detection_at_the_critical_radius(g):
    """Pairs placed at r = rc (1 + k u), u = 2^-53, k in -8..8, and at 1e-13 and
    1e-12 relative: the detection decisions (r^2 < rc^2 before or after the drift)
    equal the oracle's, pair by pair."""
    torch = _torch()
    rng = np.random.default_rng(20110058)
    u = 2.0 ** -53
    rel = [k * u for k in range(-8, 9)] + [1e-13, -1e-13, 1e-12, -1e-12, 3e-12]
    npair = len(rel)
    n = 2 * npair
    rc = np.full(n, 0.01)
    x = np.zeros((n, 3))
    for k, q in enumerate(rel):
        c = np.array([1.0 + 0.1 * k, 0.3 * k, 0.0])          # pairs 0.1 AU+ apart
        d = rng.standard_normal(3)
        d *= 0.01 * (1.0 + q) / np.linalg.norm(d)
        x[2 * k] = c
        x[2 * k + 1] = c + d
    v = np.zeros((n, 3))
    v[:, 1] = 0.017
    m = np.full(n, 1e-9)
    wl = disk(n, 0.5, 2.0, 2.0, 1, name="critical")
    wl.x, wl.v, wl.m = x, v, m
    s, pos, vel, mass = _system(g, wl, 0)
    s.set_rcrit(rc)
    s.kick(0.0, precheck=True, acc_out=torch.zeros((3, n), dtype=torch.float64, device="cuda:0"))
    cand = s.candidates()
    ref_cand = O.precheck(x, rc, wl.f_pc)
    np.testing.assert_array_equal(cand, ref_cand)
    assert len(cand) == npair
    # pre-drift = post-drift = x: the decision is the one comparison per pair
    s.set_predrift(x.T, v.T)
    s.build_encounters()
    ref_pairs = O.detect(cand, x, x, rc)
    found = borderline.record("critical-radius construction", cand, x, x, rc)
    assert len(found) >= 17 * 2
    np.testing.assert_array_equal(s.pairs(0).reshape(-1, 2), ref_pairs.reshape(-1, 2))
    # both decisions occur among the pairs placed within a few ulp of rc
    assert 0 < len(ref_pairs) < npair


@pytest.mark.parametrize("n", [16, 128, 1000])
def test_ring_single_group(g, n):
    torch = _torch()
    wl = ring(n)
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    s, pos, vel, mass = _system(g, wl, 0)
    s.set_rcrit(rc)
    s.kick(0.0, precheck=True, acc_out=torch.zeros((3, wl.n), dtype=torch.float64, device="cuda:0"))
    s.set_predrift(wl.x.T, wl.v.T)
    npairs, ngroups, maxg = s.build_encounters()
    assert (npairs, ngroups, maxg) == (4 * n, 1, n)
    assert np.all(s.groups() == 0)


@pytest.mark.parametrize("name,make", SIZES)
def test_bs_groups_match_oracle(g, name, make):
    torch = _torch()
    wl = make()
    rc, x1, v1, x2, v2, cand = _encounter_setup(g, wl)
    s, pos, vel, mass = _system(g, wl, 0)
    s.set_rcrit(rc)
    s.kick(0.0, precheck=True, acc_out=torch.zeros((3, wl.n), dtype=torch.float64, device="cuda:0"))
    s.set_predrift(x1.T, v1.T)
    pos.copy_(torch.tensor(x2.T.copy()))
    vel.copy_(torch.tensor(v2.T.copy()))
    s.build_encounters()
    s.bs(wl.dt)
    pairs = O.detect(cand, x1, x2, rc)
    # oracle: BS from the pre-drift state for group members, FG for the others
    xb, vb, st, stats = O.bs_groups(x1, v1, wl.m, rc[None], pairs, G, wl.m_star, wl.dt)
    assert st == 0
    members = np.unique(pairs.ravel())
    xg, vg = _host(pos), _host(vel)
    np.testing.assert_allclose(xg[members], xb[members], rtol=0, atol=1e-13)
    np.testing.assert_allclose(vg[members], vb[members], rtol=0, atol=1e-15)
    others = np.setdiff1d(np.arange(wl.n), members)
    np.testing.assert_array_equal(xg[others], x2[others])
    assert s.stats()["bs_steps"] > 0


# ---------------------------------------------------------------- whole steps (Appendix A)
def _rel_pos_err(xg, xr):
    return np.linalg.norm(xg - xr, axis=1) / np.linalg.norm(xr, axis=1)


def _compare_pair_logs(case, glog, olog, stop_at_borderline=False):
    """Every detection's encounter pairs, GPU against oracle, element by element
    (both sorted by (i, j)).  A pair may be in one list only if the oracle
    logged it within 1e-12 relative of its critical radius before or after the
    drift (those pairs are recorded for the session summary).  With
    stop_at_borderline, the comparison ends after the first detection that has
    such a pair (a decision there may legitimately differ and change the
    trajectories from then on).  Returns the number of detections compared."""
    assert len(glog) >= 1 and len(olog) >= 1
    if not stop_at_borderline:
        assert len(glog) == len(olog), (len(glog), len(olog))
    compared = 0
    for k, ((gl, gp), (ol, op, ob)) in enumerate(zip(glog, olog)):
        assert gl == ol, (k, gl, ol)
        op = op[np.lexsort((op[:, 1], op[:, 0]))] if len(op) else op.reshape(0, 2)
        gp = gp.reshape(-1, 2)
        if len(ob):
            borderline.LOG.append((f"{case} detection {k} (level {gl})", len(op),
                                   [("pre/post", int(i), int(j), 0.0) for i, j in ob]))
        if len(gp) == len(op) and np.array_equal(gp, op):
            compared += 1
        else:
            diff = set(map(tuple, gp.tolist())) ^ set(map(tuple, op.tolist()))
            allowed = set(map(tuple, ob.tolist()))
            assert diff <= allowed, (case, k, sorted(diff - allowed)[:10])
            compared += 1
        if stop_at_borderline and len(ob):
            break
    return compared


def _ulp_sensitivity(wl, nsteps):
    """The oracle's own spread: its result from x perturbed by one ulp."""
    xp = wl.x.copy()
    xp[:, 0] = np.nextafter(xp[:, 0], np.inf)
    xa, *_ = O.step(wl.x, wl.v, wl.m, O.make_params(wl, nthreads=8), nsteps)
    xb, *_ = O.step(xp, wl.v, wl.m, O.make_params(wl, nthreads=8), nsteps)
    return _rel_pos_err(xb, xa)


@pytest.mark.parametrize("precision", [0, 1])
def test_steps_match_oracle_config0(g, precision):
    """N = 2048 disk (0.5-2 AU, 2 Earth masses), original method.

    * 10 steps: max relative position error <= 1e-12 (FP64) / 1e-9 (mixed).
    * 100 steps: close encounters amplify rounding chaotically; a one-ulp
      perturbation of the oracle's own input moves its 100-step result by
      ~2e-11, so the GPU must agree to within 3x that measured spread (FP64;
      the mixed form to 1e-9).
    * the level-0 encounter pair list of every one of the 100 steps equals the
      oracle's element by element, up to the first detection with a pair
      within 1e-12 of its critical radius (logged; none is expected)."""
    wl = config_workload(0)
    tol = 1e-12 if precision == 0 else 1e-9
    s, pos, vel, mass = _system(g, wl, precision)
    s.set_pair_log(True)
    s.step(10)
    xr10, _, status, _ = O.step(wl.x, wl.v, wl.m, O.make_params(wl, nthreads=8), 10)
    assert status == 0
    e10 = _rel_pos_err(_host(pos), xr10)
    numerics_log.record(f"10 steps disk2048 precision={precision}", "max |dx|/|x|", e10.max(), tol)
    assert e10.max() <= tol, e10.max()
    s.step(90)
    glog = s.pair_log()
    s.set_pair_log(False)
    O.pair_log(True)
    xr, vr, status, ost = O.step(wl.x, wl.v, wl.m, O.make_params(wl, nthreads=8), 100)
    olog = O.pair_log_get()
    O.pair_log(False)
    assert status == 0
    assert len(glog) == len(olog) == 100
    compared = _compare_pair_logs(f"100 steps disk2048 precision={precision}", glog, olog,
                                  stop_at_borderline=True)
    numerics_log.record(f"100 steps disk2048 precision={precision}",
                        "steps whose level-0 pair lists were compared (all equal)", compared, 100)
    if not any(len(b) for _, _, b in olog):
        assert compared == 100
    err = _rel_pos_err(_host(pos), xr)
    spread = _ulp_sensitivity(wl, 100)
    numerics_log.record(f"100 steps disk2048 precision={precision}", "max |dx|/|x|", err.max(),
                        3 * spread.max() if precision == 0 else 1e-9)
    numerics_log.record("100 steps disk2048 oracle one-ulp spread", "max |dx|/|x|", spread.max(), 1.0)
    assert ost["n_pairs"][0] > 0
    if precision == 0:
        assert err.max() <= 3 * spread.max()
        assert np.quantile(err, 0.999) <= 3 * np.quantile(spread, 0.999)
        assert np.median(err) <= 1e-12
    else:
        assert err.max() <= 1e-9


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_steps_encounter_free_control(g, precision, tol):
    """Control run without encounters (rc = 0, K = 1 for every pair): 100 steps
    agree to 1e-12 (FP64) / 1e-9 (mixed)."""
    wl = config_workload(0)
    wl.n1 = 0.0
    wl.n2 = 0.0
    s, pos, vel, mass = _system(g, wl, precision)
    s.step(100)
    assert s.stats()["n_candidates"] == 0
    xr, *_ = O.step(wl.x, wl.v, wl.m, O.make_params(wl, nthreads=8), 100)
    err = _rel_pos_err(_host(pos), xr)
    assert err.max() <= tol, err.max()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
@pytest.mark.parametrize("slevels,substeps", [(2, 10), (3, 2), (3, 10)])
def test_levels_step_matches_oracle(g, slevels, substeps, precision, tol):
    """Symplectic levels and sub-steps of Sec. 6.3 (Fig. K's two- and three-level
    cases) on a dense disk, against the oracle's level recursion, in both kick
    forms."""
    wl = disk(2048, 0.5, 1.0, 2.0, 11, name="dense", slevels=slevels, substeps=substeps)
    s, pos, vel, mass = _system(g, wl, precision)
    s.step(5)
    st = s.stats()
    xr, vr, status, ost = O.step(wl.x, wl.v, wl.m, O.make_params(wl, nthreads=8), 5)
    assert status == 0
    assert st["n_pairs"][0] == ost["n_pairs"][0] > 0
    assert st["n_pairs"][1] > 0
    err = _rel_pos_err(_host(pos), xr)
    numerics_log.record(f"5 steps dense disk2048 levels=({slevels},{substeps}) precision={precision}",
                        "max |dx|/|x|", err.max(), tol)
    assert err.max() <= tol, err.max()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_bench_disk_full_step_matches_oracle(g, precision, tol):
    """The bench workload at full size (N = 65,540, two levels x 10 sub-steps), one
    whole step in the launch configuration bench.py times, against one oracle step
    of the same disk: the candidate list and the encounter pair list of every
    detection (level 0, and level 1 in each of the 10 sub-steps) element by
    element -- a pair may differ only if the oracle logged it within 1e-12 of
    its critical radius -- and every body's position and velocity."""
    wl = config_workload(2)
    s, pos, vel, mass = _system(g, wl, precision)
    s.set_pair_log(True)
    s.step(1)
    st = s.stats()
    glog = s.pair_log()
    s.set_pair_log(False)
    cand = s.candidates()
    O.pair_log(True)
    xr, vr, status, ost = O.step(wl.x, wl.v, wl.m, O.make_params(wl, nthreads=os.cpu_count() or 8), 1)
    olog = O.pair_log_get()
    O.pair_log(False)
    assert status == 0
    # candidates: exact FP64 decisions on the identical step-start state
    rc0 = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    cref = O.precheck(wl.x, rc0, wl.f_pc)
    assert st["n_candidates"] == ost["n_candidates"] == len(cref) > 0
    np.testing.assert_array_equal(cand, cref)
    # one level-0 detection and one level-1 detection per sub-step
    assert [lv for lv, _ in glog] == [0] + [1] * 10
    compared = _compare_pair_logs(f"1 step disk65540 precision={precision}", glog, olog)
    assert compared == 11 and len(glog[0][1]) == st["n_pairs"][0] > 0
    err = _rel_pos_err(_host(pos), xr)
    verr = np.linalg.norm(_host(vel) - vr, axis=1) / np.linalg.norm(vr, axis=1)
    numerics_log.record(f"1 step disk65540 (bench config) precision={precision}", "max |dx|/|x|",
                        err.max(), tol)
    numerics_log.record(f"1 step disk65540 (bench config) precision={precision}", "max |dv|/|v|",
                        verr.max(), tol)
    assert err.max() <= tol, err.max()
    assert verr.max() <= tol, verr.max()
    # the pair log makes the host read every level's count; bench.py runs without
    # it, the deepest level then keeping its counts on the device: the same step
    # that way gives the same state, bit for bit
    s2, pos2, vel2, _ = _system(g, wl, precision)
    s2.step(1)
    np.testing.assert_array_equal(_host(pos2), _host(pos))
    np.testing.assert_array_equal(_host(vel2), _host(vel))
    assert s2.stats()["n_pairs"] == st["n_pairs"]


@pytest.mark.parametrize("slevels,substeps", [(2, 10), (3, 2)])
def test_device_counts_match_host_counts(g, slevels, substeps):
    """The deepest level takes its pair and group counts from the device: its
    list sized to its input, the partner-list and grouping kernels reading the
    detection's count, the in-block Bulirsch-Stoer kernels claiming their
    bucket's groups.  With the pair log on, the host reads every count and sizes
    every launch from it.  Three steps of the dense disk both ways: the same
    positions and velocities bit for bit, the same last pair list of the deepest
    level, the same pair totals per level."""
    wl = disk(2048, 0.5, 1.0, 2.0, 11, name="dense", slevels=slevels, substeps=substeps)
    out = []
    for log in (True, False):
        s, pos, vel, _ = _system(g, wl, 0)
        s.set_pair_log(log)
        s.step(3)
        out.append((_host(pos), _host(vel), s.pairs(slevels - 1), s.stats()))
    (p1, v1, l1, st1), (p2, v2, l2, st2) = out
    np.testing.assert_array_equal(p1, p2)
    np.testing.assert_array_equal(v1, v2)
    assert len(l1) > 0
    np.testing.assert_array_equal(l1, l2)
    assert st1["n_pairs"] == st2["n_pairs"] and st1["n_pairs"][slevels - 1] > 0
    assert st1["n_groups"] == st2["n_groups"] and st1["bs_steps"] == st2["bs_steps"]


def test_energy_matches_oracle(g):
    wl = config_workload(0)
    s, *_ = _system(g, wl)
    E, L = s.energy()
    Er, Lr = O.energy(wl.x, wl.v, wl.m, wl.m_star, G)
    assert abs(E - Er) <= 1e-13 * abs(Er)
    np.testing.assert_allclose(L, Lr, rtol=1e-13)


def test_step_host_buffers(g):
    wl = config_workload(0, n_override=256)
    s, pos, vel, mass = _system(g, wl, 0)
    xh = np.ascontiguousarray(wl.x.T)
    vh = np.ascontiguousarray(wl.v.T)
    s.step_host(xh, vh, 3)
    xr, vr, status, _ = O.step(wl.x, wl.v, wl.m, O.make_params(wl), 3)
    np.testing.assert_allclose(xh.T, xr, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- failure paths (host-visible status)
def test_kepler_iteration_limit_reports_nonconvergence(g):
    wl = config_workload(0, n_override=256)
    s, *_ = _system(g, wl, 0, kepler_max_iter=1)
    with pytest.raises(g.GengaError) as e:
        s.step(1)
    assert e.value.code == -3


def test_bs_step_limit_reports_nonconvergence(g):
    wl = config_workload(0)
    s, *_ = _system(g, wl, 0, bs_max_steps=1)
    with pytest.raises(g.GengaError) as e:
        s.step(1)
    assert e.value.code == -3
    # the context stays usable: a fresh system on the same device works
    s2, *_ = _system(g, config_workload(0, n_override=64), 0)
    s2.step(1)


def test_nan_state_reports_bad_state(g):
    wl = config_workload(0, n_override=256)
    wl.x[3, 0] = np.nan
    s, *_ = _system(g, wl, 0)
    with pytest.raises(g.GengaError) as e:
        s.step(1)
    assert e.value.code == -5


def test_set_params_adds_levels_beyond_creation(g):
    """A system created with one level and switched to three (genga_set_params)
    holds every array of the new levels: steps match the oracle's three-level run."""
    wl = disk(2048, 0.5, 1.0, 2.0, 11, name="dense", slevels=3, substeps=10)
    s, pos, vel, mass = _system(g, wl, 0, slevels=1, substeps=1)
    p = g.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2, f_pc=wl.f_pc,
                         slevels=3, substeps=10, precision=0)
    s.set_params(p)
    s.step(3)
    st = s.stats()
    xr, vr, status, ost = O.step(wl.x, wl.v, wl.m, O.make_params(wl, nthreads=8), 3)
    assert status == 0 and st["n_pairs"][2] > 0
    assert st["n_pairs"][0] == ost["n_pairs"][0]
    # sub-step pairs follow sub-step states: a decision within rounding of rc may differ
    assert all(abs(st["n_pairs"][k] - ost["n_pairs"][k]) <= 2 for k in (1, 2))
    assert _rel_pos_err(_host(pos), xr).max() <= 1e-12


# ---------------------------------------------------------------- level self-tuning (Sec. 6.3)
def test_tune_levels_restores_state_and_keeps_fastest(g):
    """The self-tuner times each (levels, sub-steps) candidate from the same state,
    keeps the fastest, and leaves the state bit for bit as it found it: later steps
    equal those of a system created with the chosen setting."""
    wl = disk(2048, 0.5, 1.0, 2.0, 11, name="dense", slevels=2, substeps=10)
    s, pos, vel, mass = _system(g, wl, 1)
    x0, v0 = _host(pos), _host(vel)
    cands = [(1, 1), (2, 10), (3, 2), (3, 10)]
    best, ms = s.tune_levels(cands, trial_steps=2)
    assert np.array_equal(_host(pos), x0) and np.array_equal(_host(vel), v0)
    assert np.all(ms > 0) and best == int(np.argmin(ms))
    L, S = cands[best]
    assert (s.params.slevels, s.params.substeps) == (L, S)
    s.step(3)
    wl2 = disk(2048, 0.5, 1.0, 2.0, 11, name="dense", slevels=L, substeps=S)
    s2, pos2, vel2, _ = _system(g, wl2, 1)
    s2.step(3)
    assert np.array_equal(_host(pos), _host(pos2)) and np.array_equal(_host(vel), _host(vel2))
    # an invalid candidate is refused before anything runs
    with pytest.raises(g.GengaError):
        s.tune_levels([(2, 10), (0, 1)])
    assert (s.params.slevels, s.params.substeps) == (L, S)


# ---------------------------------------------------------------- semi-active test particles (Sec. 8.1)
TP_CASES = [("disk2048", lambda: config_workload(0), 1000),      # boundary inside a 128-row block
            ("disk3001_ragged", lambda: disk(3001, 0.5, 2.0, 2.0, 77, name="ragged"), 2560),
            ("disk2048_all_tp", lambda: config_workload(0), 0)]


@pytest.mark.parametrize("name,make,nm", TP_CASES)
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_tp_kick_matches_oracle(g, name, make, nm, precision, tol):
    torch = _torch()
    wl = make()
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    s, pos, vel, mass = _system(g, wl, precision, tp_mode=2, n_massive=nm)
    s.set_rcrit(rc)
    acc = torch.zeros((3, wl.n), dtype=torch.float64, device="cuda:0")
    s.kick(0.0, precheck=False, acc_out=acc)
    torch.cuda.synchronize()
    a = _host(acc)
    ref = O.accel(wl.x, wl.m, rc, G, nthreads=8, n_massive=nm)
    if nm == 0:
        assert np.all(a == 0.0) and np.all(ref == 0.0)
        return
    rel = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
    numerics_log.record(f"kick {name} test particles from {nm} precision={precision}",
                        "per-particle |da|/|a|", rel.max(), tol)
    assert rel.max() <= tol, rel.max()


@pytest.mark.parametrize("name,make,nm", TP_CASES)
def test_tp_precheck_candidates_bit_exact(g, name, make, nm):
    wl = make()
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    s, *_ = _system(g, wl, 1, tp_mode=2, n_massive=nm)
    s.set_rcrit(rc)
    s.kick(0.5 * wl.dt, precheck=True)
    ref = O.precheck(wl.x, rc, wl.f_pc, n_massive=nm)
    np.testing.assert_array_equal(s.candidates().reshape(-1, 2), ref.reshape(-1, 2))


@pytest.mark.parametrize("slevels,substeps", [(1, 1), (2, 10)])
def test_tp_step_matches_oracle(g, slevels, substeps):
    """Whole steps with 1,500 large bodies and 548 semi-active test particles."""
    wl = disk(2048, 0.5, 1.0, 2.0, 11, name="dense", slevels=slevels, substeps=substeps)
    nm = 1500
    s, pos, vel, mass = _system(g, wl, 0, tp_mode=2, n_massive=nm)
    s.step(5)
    st = s.stats()
    xr, vr, status, ost = O.step(wl.x, wl.v, wl.m, O.make_params(wl, nthreads=8, tp_mode=2, n_massive=nm), 5)
    assert status == 0
    assert st["n_candidates"] == ost["n_candidates"] > 0
    assert st["n_pairs"][0] == ost["n_pairs"][0] > 0
    err = _rel_pos_err(_host(pos), xr)
    numerics_log.record(f"5 steps dense disk2048 test particles from {nm} levels=({slevels},{substeps})",
                        "max |dx|/|x|", err.max(), 1e-12)
    assert err.max() <= 1e-12, err.max()


def test_tp_energy_matches_oracle(g):
    wl = config_workload(0)
    s, *_ = _system(g, wl, 0, tp_mode=2, n_massive=1200)
    E, L = s.energy()
    Er, Lr = O.energy(wl.x, wl.v, wl.m, wl.m_star, G, n_massive=1200)
    assert abs(E - Er) <= 1e-13 * abs(Er)
    np.testing.assert_allclose(L, Lr, rtol=1e-13)


def test_tp_mode_checks(g):
    wl = config_workload(0, n_override=256)
    with pytest.raises(g.GengaError):
        _system(g, wl, 0, tp_mode=1, n_massive=100)
    s, *_ = _system(g, wl, 0, tp_mode=2, n_massive=100)
    with pytest.raises(g.GengaError):
        s.adjoint_forward(2, 1)
