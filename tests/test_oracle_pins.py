"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here checks the oracle against something other than itself: closed
forms, conservation laws, brute force on tiny inputs, an independent
high-accuracy integration of the same equations of motion, or a textbook
solution reached by a different route (classical anomalies instead of
universal variables).
"""
import numpy as np
import pytest

import oracle as O
from tests import twobody
from workloads import G_GAUSS, M_EARTH, config_workload, disk, ring

G = G_GAUSS


# ---------------------------------------------------------------- changeover (Sec. 6.3, fn.)
def test_changeover_outside_band_is_exactly_0_or_1():
    rc = 0.037
    for r in [0.0, 1e-9, 0.05 * rc, 0.1 * rc]:
        assert O.changeover(r, rc) == 0.0
    for r in [rc, 1.0000001 * rc, 2 * rc, 1e3]:
        assert O.changeover(r, rc) == 1.0


def test_changeover_symmetry_midpoint_smoothness_monotone():
    rc = 1.0
    ys = np.linspace(0.0, 1.0, 2001)
    K = np.array([O.changeover(0.1 + 0.9 * y, rc) for y in ys])
    Kr = np.array([O.changeover(0.1 + 0.9 * (1 - y), rc) for y in ys])
    assert np.all(K >= 0) and np.all(K <= 1)
    # K(y) + K(1-y) = 1 (up to the rounding of y from r)
    assert np.max(np.abs(K + Kr - 1.0)) < 1e-14
    # K(1/2) = 1/2
    assert abs(O.changeover(0.55, rc) - 0.5) < 1e-15
    assert np.all(np.diff(K) >= 0)
    # smooth switch: zero slope at both ends (K ~ y^2 near 0)
    for y in [1e-3, 1e-4]:
        k0 = O.changeover(0.1 + 0.9 * y, rc)
        k1 = O.changeover(0.1 + 0.9 * (1 - y), rc)
        assert k0 / y < 2.1 * y and (1 - k1) / y < 2.1 * y


# ---------------------------------------------------------------- Eq. rcrit
def test_rcrit_hand_values():
    x = np.array([[1.0, 0.0, 0.0], [0.0, 5.0, 0.0], [3.0, 4.0, 0.0]])
    v = np.array([[0.0, 0.0172, 0.0], [0.001, 0.0, 0.0], [0.003, 0.004, 0.0]])
    m = np.array([3e-6, 3e-3, 3e-9])
    rc = O.rcrit(x, v, m, 1.0, 6.0875, 3.0, 0.4)
    # body 0: 3 R_H = 0.03 < 0.4*6.0875*0.0172 = 0.041882
    # body 1: 3 R_H = 3*5*0.1 = 1.5 > 0.4*6.0875*0.001
    # body 2: 3 R_H = 3*5*0.001 = 0.015 > 0.4*6.0875*0.005 = 0.012175
    np.testing.assert_allclose(rc, [0.041882, 1.5, 0.015], rtol=1e-14)


# ---------------------------------------------------------------- Eq. Hb kick
def test_kick_two_body_closed_form():
    x = np.array([[1.0, 0.0, 0.0], [1.0, 2.0, 0.0]])
    m = np.array([1e-5, 3e-5])
    rc = np.array([1e-6, 1e-6])         # far outside rc: K = 1
    a = O.accel(x, m, rc, G)
    np.testing.assert_allclose(a[0], [0.0, G * 3e-5 / 4.0, 0.0], rtol=1e-15, atol=0)
    np.testing.assert_allclose(a[1], [0.0, -G * 1e-5 / 4.0, 0.0], rtol=1e-15, atol=0)


def _random_cluster(n, seed, spread=0.05):
    rng = np.random.default_rng(seed)
    x = np.array([1.0, 0.0, 0.0]) + spread * rng.standard_normal((n, 3))
    m = rng.uniform(1e-8, 1e-6, n)
    rc = rng.uniform(0.01, 0.08, n)
    return x, m, rc


def test_kick_conserves_momentum_and_angular_momentum():
    x, m, rc = _random_cluster(60, 1)
    a = O.accel(x, m, rc, G)
    K = np.array([[O.changeover(np.linalg.norm(x[j] - x[i]), max(rc[i], rc[j])) if i != j else 0
                   for j in range(60)] for i in range(60)])
    assert 0.0 < K.min() + 1 and np.any((K > 0) & (K < 1)), "cluster must straddle the band"
    F = m[:, None] * a
    scale = np.abs(F).sum(axis=0).max()
    assert np.abs(F.sum(axis=0)).max() < 1e-14 * scale
    T = np.cross(x, F)
    assert np.abs(T.sum(axis=0)).max() < 1e-13 * np.abs(T).sum(axis=0).max()


def test_kick_without_changeover_equals_direct_sum_longdouble():
    x, m, _ = _random_cluster(50, 2, spread=0.3)
    rc = np.full(50, 1e-12)              # every pair is far outside rc: K = 1
    a = O.accel(x, m, rc, G)
    X = x.astype(np.longdouble)
    d = X[None, :, :] - X[:, None, :]
    r2 = (d * d).sum(axis=2)
    np.fill_diagonal(r2, 1)
    w = m.astype(np.longdouble)[None, :] / (r2 * np.sqrt(r2))
    np.fill_diagonal(w, 0)
    ref = np.longdouble(G) * (w[:, :, None] * d).sum(axis=1)
    np.testing.assert_allclose(a, ref.astype(np.float64), rtol=1e-13, atol=0)


def test_kick_pair_inside_inner_radius_contributes_nothing():
    x = np.array([[1.0, 0, 0], [1.001, 0, 0], [1.5, 0.5, 0]])
    m = np.array([1e-6, 2e-6, 3e-6])
    rc = np.array([0.1, 0.1, 1e-9])      # pair (0,1): r = 0.001 < 0.1 rc -> K = 0
    a = O.accel(x, m, rc, G)
    d = x[2] - x[0]
    ref0 = G * m[2] * d / np.linalg.norm(d) ** 3
    np.testing.assert_allclose(a[0], ref0, rtol=1e-15)


def test_kick_velocity_update():
    x, m, rc = _random_cluster(20, 3)
    v = np.zeros_like(x)
    v2 = O.kick(x, v, m, rc, G, 0.5)
    np.testing.assert_allclose(v2, 0.5 * O.accel(x, m, rc, G), rtol=1e-15)


# ---------------------------------------------------------------- pre-check / detection / grouping
def _brute_pairs(x, rc, fac):
    n = len(rc)
    out = []
    for i in range(n):
        for j in range(i + 1, n):
            d = x[j] - x[i]
            if np.sqrt((d * d).sum()) < fac * max(rc[i], rc[j]):
                out.append((i, j))
    return np.array(out, dtype=np.uint32).reshape(-1, 2)


def test_precheck_brute_force():
    x, _, rc = _random_cluster(80, 4)
    cand = O.precheck(x, rc, 4.0)
    assert len(cand) > 0
    np.testing.assert_array_equal(cand, _brute_pairs(x, rc, 4.0))


def test_detect_brute_force_and_order():
    x, _, rc = _random_cluster(80, 5)
    rng = np.random.default_rng(7)
    xpost = x + 0.02 * rng.standard_normal(x.shape)
    cand = O.precheck(x, rc, 4.0)
    enc = O.detect(cand, x, xpost, rc)
    ref = []
    for i, j in cand:
        rcij = max(rc[i], rc[j])
        if (np.linalg.norm(x[j] - x[i]) < rcij) or (np.linalg.norm(xpost[j] - xpost[i]) < rcij):
            ref.append((i, j))
    np.testing.assert_array_equal(enc, np.array(ref, dtype=np.uint32).reshape(-1, 2))
    keys = enc[:, 0].astype(np.uint64) << 32 | enc[:, 1]
    assert np.all(np.diff(keys.astype(np.int64)) > 0)


def test_group_brute_force_components():
    rng = np.random.default_rng(9)
    n = 50
    pairs = set()
    while len(pairs) < 30:
        i, j = sorted(rng.integers(0, n, 2))
        if i != j:
            pairs.add((int(i), int(j)))
    pairs = np.array(sorted(pairs), dtype=np.uint32)
    lab = O.group(n, pairs)
    # components by depth-first search
    adj = {i: set() for i in range(n)}
    for i, j in pairs:
        adj[int(i)].add(int(j))
        adj[int(j)].add(int(i))
    seen = {}
    for s in range(n):
        if s in seen or not adj[s]:
            continue
        comp, stack = [], [s]
        seen[s] = True
        while stack:
            u = stack.pop()
            comp.append(u)
            for w in adj[u]:
                if w not in seen:
                    seen[w] = True
                    stack.append(w)
        for u in comp:
            assert lab[u] == min(comp)
    for i in range(n):
        if not adj[i]:
            assert lab[i] == -1


@pytest.mark.parametrize("n", [8, 12, 16, 64, 128])
def test_ring_is_one_group_with_eight_partners(n):
    """Sec. 6.2 ring test: every body meets eight neighbours (all others for
    N < 16) and the ring forms a single close-encounter group."""
    wl = ring(n)
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    cand = O.precheck(wl.x, rc, wl.f_pc)
    enc = O.detect(cand, wl.x, wl.x, rc)
    expect = n * (n - 1) // 2 if n < 16 else 4 * n
    assert len(enc) == expect
    lab = O.group(n, enc)
    assert np.all(lab == 0)
    deg = np.bincount(enc.ravel(), minlength=n)
    assert np.all(deg == (n - 1 if n < 16 else 8))


# ---------------------------------------------------------------- Eq. Hc
def test_hc_uniform_shift():
    wl = config_workload(0, n_override=64)
    dt_half = 3.0
    x1 = O.hc(wl.x, wl.v, wl.m, wl.m_star, dt_half)
    P = (wl.m[:, None] * wl.v).sum(axis=0)
    shift = x1 - wl.x
    # the shift is recovered as a difference of O(1) numbers: 2 ulp of |x| each
    np.testing.assert_allclose(shift, np.broadcast_to(dt_half * P / wl.m_star, shift.shape),
                               rtol=0, atol=4 * np.finfo(float).eps * np.abs(wl.x).max())
    d0 = wl.x[:, None, :] - wl.x[None, :, :]
    d1 = x1[:, None, :] - x1[None, :, :]
    assert np.abs(d1 - d0).max() <= 8 * np.finfo(float).eps * 2.0


# ---------------------------------------------------------------- Eq. Ha Kepler drift
def _orbit(a, e, inc, Om, om, M, mu):
    from workloads.disk import elements_to_cartesian
    x, v = elements_to_cartesian(np.array([a]), np.array([e]), np.array([inc]), np.array([Om]),
                                 np.array([om]), np.array([M]), mu)
    return x[0], v[0]


@pytest.mark.parametrize("e", [0.0, 0.01, 0.3, 0.7, 0.95])
@pytest.mark.parametrize("dt", [0.3, 6.0875, 200.0, -50.0])
def test_drift_matches_eccentric_anomaly_solution(e, dt):
    mu = G
    x0, v0 = _orbit(1.3, e, 0.2, 0.4, 1.1, 2.0, np.array([mu]))
    x1, v1, fails = O.drift(x0[None], v0[None], mu, dt)
    assert fails == 0
    xr, vr = twobody.propagate(x0, v0, mu, dt)
    np.testing.assert_allclose(x1[0], xr, rtol=0, atol=2e-13 * np.linalg.norm(xr) * max(1, abs(dt) / 100))
    np.testing.assert_allclose(v1[0], vr, rtol=0, atol=2e-13 * np.linalg.norm(vr) * max(1, abs(dt) / 100))


@pytest.mark.parametrize("e", [1.5, 3.0])
def test_drift_matches_hyperbolic_anomaly_solution(e):
    mu = G
    q = 0.5
    a = -q / (e - 1)
    # state at periapsis, then integrate from a point before it
    r = q
    vp = np.sqrt(mu * (2 / r - 1 / a))
    x0 = np.array([r, 0.0, 0.0])
    v0 = np.array([0.0, vp, 0.0])
    for dt in [5.0, 40.0, -30.0]:
        x1, v1, fails = O.drift(x0[None], v0[None], mu, dt)
        assert fails == 0
        xr, vr = twobody.propagate(x0, v0, mu, dt)
        np.testing.assert_allclose(x1[0], xr, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(v1[0], vr, rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("e", [0.999999, 1.0, 1.000001])
def test_drift_near_parabolic_invariants(e):
    mu = G
    q = 0.3
    r = q
    vp = np.sqrt(mu * (1 + e) / q)
    x0 = np.array([r, 0.0, 0.0])
    v0 = np.array([0.0, vp, 0.0])
    x1, v1, fails = O.drift(x0[None], v0[None], mu, 30.0)
    assert fails == 0
    E0, h0, A0 = twobody.invariants(x0, v0, mu)
    E1, h1, A1 = twobody.invariants(x1[0], v1[0], mu)
    assert abs(float(E1 - E0)) < 1e-14 * float(np.abs(np.dot(v0, v0)))
    assert np.abs((h1 - h0).astype(float)).max() < 1e-14 * float(np.linalg.norm(h0.astype(float)))
    assert np.abs((A1 - A0).astype(float)).max() < 1e-13 * mu


def test_drift_invariants_reversibility_and_composition():
    wl = config_workload(0, n_override=256)
    mu = G * wl.m_star
    x1, v1, f1 = O.drift(wl.x, wl.v, mu, 6.0875)
    assert f1 == 0
    for k in range(0, 256, 17):
        E0, h0, A0 = twobody.invariants(wl.x[k], wl.v[k], mu)
        E1, h1, A1 = twobody.invariants(x1[k], v1[k], mu)
        assert abs(float((E1 - E0) / E0)) < 1e-14
        assert np.abs((h1 - h0).astype(float)).max() < 1e-14 * float(np.linalg.norm(h0.astype(float)))
        assert np.abs((A1 - A0).astype(float)).max() < 1e-13 * mu
    xb, vb, _ = O.drift(x1, v1, mu, -6.0875)
    np.testing.assert_allclose(xb, wl.x, rtol=0, atol=1e-14)
    np.testing.assert_allclose(vb, wl.v, rtol=0, atol=1e-16)
    xa, va, _ = O.drift(wl.x, wl.v, mu, 2.5)
    xab, vab, _ = O.drift(xa, va, mu, 3.5875)
    np.testing.assert_allclose(xab, x1, rtol=0, atol=1e-14)
    np.testing.assert_allclose(vab, v1, rtol=0, atol=1e-16)


def test_drift_iteration_limit_reports_failure():
    wl = config_workload(0, n_override=8)
    _, _, fails = O.drift(wl.x, wl.v, G, 6.0875, max_iter=1)
    assert fails == 8


# ---------------------------------------------------------------- Bulirsch-Stoer (Sec. 6.1)
@pytest.mark.parametrize("tol", [1e-15, 1e-13])
def test_bs_pure_two_body_without_star(tol):
    """m_star = 0 and K = 0: the group ODE is the two-body problem.  The error
    control holds each step's error near tol relative to the state's scale
    (coordinates ~1 AU here), so the bounds follow the tolerance."""
    m = np.array([3e-6, 1e-6])
    x = np.array([[1.0, 0.0, 0.0], [1.01, 0.0, 0.0]])
    mu_rel = G * m.sum()
    vrel = np.array([0.0, 1.2 * np.sqrt(mu_rel / 0.01), 0.0])   # bound, e ~ 0.44
    v = np.zeros((2, 3))
    v[0] = -m[1] / m.sum() * vrel
    v[1] = m[0] / m.sum() * vrel
    rc = np.array([[1e3, 1e3]])                                   # r << 0.1 rc: K = 0
    pairs = np.array([[0, 1]], dtype=np.uint32)
    dt = 30.0
    x1, v1, st, stats = O.bs_groups(x, v, m, rc, pairs, G, 0.0, dt, tol=tol)
    assert st == 0 and stats["n_groups"] == 1
    xr, vr = twobody.propagate(x[1] - x[0], vrel, mu_rel, dt)
    com = (m[:, None] * x).sum(axis=0) / m.sum()
    k = max(1.0, tol / 1e-14)
    np.testing.assert_allclose(x1[1] - x1[0], xr, rtol=0, atol=k * 1e-12 * 0.01)
    np.testing.assert_allclose(v1[1] - v1[0], vr, rtol=0, atol=k * 1e-12 * np.linalg.norm(vrel))
    np.testing.assert_allclose((m[:, None] * x1).sum(axis=0) / m.sum(), com, rtol=0, atol=2e-14)


@pytest.mark.parametrize("tol", [1e-15, 1e-13])
def test_bs_star_term_is_kepler(tol):
    """A massive body paired with a massless partner follows its exact Kepler
    orbit, to within the error control's tolerance."""
    m = np.array([1e-6, 0.0])
    x0, v0 = _orbit(1.0, 0.2, 0.1, 0.3, 0.5, 1.0, np.array([G]))
    # a massless partner passing by on a hyperbolic flyby
    x = np.array([x0, x0 + np.array([0.004, 0.0, 0.0])])
    v = np.array([v0, v0 + np.array([0.0, 0.001, 0.0])])
    rc = np.array([[0.05, 0.05]])
    pairs = np.array([[0, 1]], dtype=np.uint32)
    x1, v1, st, _ = O.bs_groups(x, v, m, rc, pairs, G, 1.0, 6.0875, tol=tol)
    assert st == 0
    xr, vr = twobody.propagate(x0, v0, G, 6.0875)
    k = max(1.0, tol / 1e-14)
    np.testing.assert_allclose(x1[0], xr, rtol=0, atol=k * 1e-14)
    np.testing.assert_allclose(v1[0], vr, rtol=0, atol=k * 2e-14 * np.linalg.norm(vr))


def test_bs_converges_as_tolerance_tightens():
    """The achieved error stays within the requested tolerance (relative to the
    state's scale) and vanishes as the tolerance tightens."""
    m = np.array([3e-6, 3e-6])
    x0, v0 = _orbit(1.0, 0.01, 0.0, 0.0, 0.0, 0.0, np.array([G]))
    x = np.array([x0, x0 + np.array([0.0, 0.004, 0.0])])
    v = np.array([v0, v0 + np.array([0.0004, 0.0, 0.0])])
    rc = np.array([[0.03, 0.03]])
    pairs = np.array([[0, 1]], dtype=np.uint32)
    ref, _, _, _ = O.bs_groups(x, v, m, rc, pairs, G, 1.0, 6.0875, tol=1e-15)
    errs = {}
    for tol in [1e-5, 1e-7, 1e-9, 1e-11, 1e-13]:
        x1, v1, st, _ = O.bs_groups(x, v, m, rc, pairs, G, 1.0, 6.0875, tol=tol)
        assert st == 0
        errs[tol] = np.abs(x1 - ref).max()
        assert errs[tol] <= 10 * tol * np.abs(x).max() + 1e-14
    assert errs[1e-5] > 1e3 * errs[1e-11]


def test_bs_step_limit_reports_failure():
    m = np.array([3e-6, 3e-6])
    x = np.array([[1.0, 0, 0], [1.001, 0, 0]])
    v = np.array([[0, 0.0172, 0], [0, 0.0172, 0.001]])
    rc = np.array([[0.03, 0.03]])
    _, _, st, stats = O.bs_groups(x, v, m, rc, np.array([[0, 1]], dtype=np.uint32), G, 1.0,
                                  6.0875, max_steps=1)
    assert st == 2 and stats["bs_fail"] == 1


# ---------------------------------------------------------------- whole step (Appendix A)
def _reference_dhc(x, v, m, m_star, T):
    """Exact dynamics in democratic heliocentric coordinates, integrated with DOP853:
    dx_i/dt = v_i + P/m_star,  dv_i/dt = -G m_star x_i/r_i^3 + G sum_j m_j (x_j-x_i)/r_ij^3."""
    from scipy.integrate import solve_ivp
    n = len(m)

    def rhs(_, y):
        X = y[:3 * n].reshape(n, 3)
        V = y[3 * n:].reshape(n, 3)
        P = (m[:, None] * V).sum(axis=0)
        r = np.linalg.norm(X, axis=1)
        acc = -G * m_star * X / r[:, None] ** 3
        d = X[None, :, :] - X[:, None, :]
        r2 = (d * d).sum(axis=2)
        np.fill_diagonal(r2, 1.0)
        w = m[None, :] / r2 ** 1.5
        np.fill_diagonal(w, 0.0)
        acc += G * (w[:, :, None] * d).sum(axis=1)
        return np.concatenate([(V + P / m_star).ravel(), acc.ravel()])

    sol = solve_ivp(rhs, (0, T), np.concatenate([x.ravel(), v.ravel()]), method="DOP853",
                    rtol=1e-13, atol=1e-18)
    y = sol.y[:, -1]
    return y[:3 * n].reshape(n, 3), y[3 * n:].reshape(n, 3)


def _few_body(close: bool):
    m = np.array([3e-6, 5e-6, 1e-6, 2e-6, 4e-6])
    a = np.array([0.8, 1.0, 1.25, 1.5, 1.9])
    el = [(a[k], 0.02 * (k + 1), 0.01 * k, 0.3 * k, 0.7 * k, 1.3 * k) for k in range(5)]
    if close:
        # body 2 shares body 1's orbit, slightly wider and 0.025 rad ahead: the
        # pair starts inside 3 Hill radii and drifts apart
        a1, e1, i1, O1, w1, M1 = el[1]
        el[2] = (a1 + 0.004, e1, i1, O1, w1, M1 + 0.025)
    x = np.zeros((5, 3))
    v = np.zeros((5, 3))
    for k in range(5):
        xx, vv = _orbit(*el[k], np.array([G * (1 + m[k])]))
        x[k], v[k] = xx, vv
    v = v - (m[:, None] * v).sum(axis=0) / (1 + m.sum())
    return x, v, m


@pytest.mark.parametrize("close", [False, True])
def test_step_second_order_convergence(close):
    x, v, m = _few_body(close)
    T = 96.0
    xr, vr = _reference_dhc(x, v, m, 1.0, T)
    errs = []
    for nst in [16, 32, 64]:
        dt = T / nst
        # Hill-only critical radius (n2 = 0) keeps the split fixed as dt shrinks
        p = O.make_params(dt=dt, n1=3.0, n2=0.0, f_pc=4.0)
        x1, v1, st, stats = O.step(x, v, m, p, nst)
        assert st == 0
        if close:
            assert stats["n_groups"] > 0
        errs.append(np.abs(x1 - xr).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, errs


def test_step_conserves_angular_momentum_with_encounters():
    wl = config_workload(0, n_override=512)
    p = O.make_params(wl, nthreads=4)
    _, L0 = O.energy(wl.x, wl.v, wl.m, wl.m_star, G)
    x1, v1, st, stats = O.step(wl.x, wl.v, wl.m, p, 5)
    assert st == 0 and stats["n_groups"] > 0
    _, L1 = O.energy(x1, v1, wl.m, wl.m_star, G)
    assert np.abs(L1 - L0).max() < 1e-14 * 5 * np.linalg.norm(L0)


def test_step_energy_bounded_and_second_order_without_encounters():
    """Symplectic behaviour: the energy error stays bounded over 20,000 steps (no
    trend between the first and second half) and scales as dt^2."""
    E0 = None
    maxes = []
    for dt, nst in [(6.0875, 200), (6.0875 / 2, 400)]:
        x, v, m = _few_body(False)
        p = O.make_params(dt=dt, n1=3.0, n2=0.0)
        if E0 is None:
            E0, _ = O.energy(x, v, m, 1.0, G)
        errs = []
        for _ in range(100):
            x, v, st, stats = O.step(x, v, m, p, nst)
            assert st == 0 and stats["n_groups"] == 0
            E, _ = O.energy(x, v, m, 1.0, G)
            errs.append(abs((E - E0) / E0))
        errs = np.array(errs)
        assert errs[50:].max() < 1.5 * errs[:50].max()
        maxes.append(errs.max())
    assert maxes[0] < 1e-7
    assert 3.5 < maxes[0] / maxes[1] < 4.5


def test_step_levels_reduce_groups():
    """Sec. 6.3: a second level at dt/10 shrinks the BS groups."""
    wl = disk(1024, 0.5, 1.0, 2.0, 11, name="dense")
    p1 = O.make_params(wl, slevels=1, substeps=1, nthreads=4)
    p2 = O.make_params(wl, slevels=2, substeps=10, nthreads=4)
    _, _, s1, st1 = O.step(wl.x, wl.v, wl.m, p1, 1)
    x2, v2, s2, st2 = O.step(wl.x, wl.v, wl.m, p2, 1)
    assert s1 == 0 and s2 == 0
    assert st2["n_pairs"][0] == st1["n_pairs"][0] > 0
    assert st2["max_group"] < st1["max_group"]
    E0, _ = O.energy(wl.x, wl.v, wl.m, 1.0, G)
    E2, _ = O.energy(x2, v2, wl.m, 1.0, G)
    assert abs((E2 - E0) / E0) < 1e-8


# ---------------------------------------------------------------- energy (Eq. H)
def test_energy_hand_value():
    x = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    v = np.array([[0.0, 0.01, 0.0], [0.005, 0.0, 0.0]])
    m = np.array([1e-3, 2e-3])
    E, L = O.energy(x, v, m, 1.0, 1.0)
    kin = 0.5 * 1e-3 * 1e-4 + 0.5 * 2e-3 * 2.5e-5
    pot_star = -1e-3 / 1.0 - 2e-3 / 2.0
    pot_pair = -1e-3 * 2e-3 / np.sqrt(5.0)
    P = np.array([2e-3 * 0.005, 1e-3 * 0.01, 0.0])
    hc = (P @ P) / 2.0
    assert abs(E - (kin + pot_star + pot_pair + hc)) < 1e-18
    np.testing.assert_allclose(L, [0.0, 0.0, 1e-3 * 0.01 - 2e-3 * 2.0 * 0.005], rtol=1e-15)
