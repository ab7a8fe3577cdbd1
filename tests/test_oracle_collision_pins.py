"""Pins of the oracle's collisions (Sec. 7.1-7.2; reading R25).

The merger is checked against the conservation laws it must satisfy (mass,
linear momentum, total angular momentum with spins, R^3, and the two-body
energy split into centre-of-mass and relative parts), the index rule of
Sec. 7.1, and the contact time of a radial two-body infall (closed form)
within the collision precision of Sec. 7.2.
"""
import numpy as np
import pytest

import oracle as O
from workloads import G_GAUSS, config_workload, disk

G = G_GAUSS


def _pair(seed=2, mi=3e-6, mj=1e-6):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((2, 3))
    v = rng.standard_normal((2, 3)) * 0.02
    m = np.array([mi, mj])
    R = np.array([3e-5, 2e-5])
    S = rng.standard_normal((2, 3)) * 1e-12
    return x, v, m, R, S


def test_merger_conserves_what_the_paper_says():
    x, v, m, R, S = _pair()
    x1, v1, m1, R1, S1, dU, sv = O.merge(0, 1, x, v, m, R, S, G)
    ot = 1 - sv
    M = m.sum()
    assert m1[sv] == M and m1[ot] == 0.0 and R1[ot] == 0.0 and np.all(S1[ot] == 0.0)
    np.testing.assert_allclose(M * v1[sv], m[0] * v[0] + m[1] * v[1], rtol=1e-15, atol=0)
    np.testing.assert_allclose(M * x1[sv], m[0] * x[0] + m[1] * x[1], rtol=1e-15, atol=0)
    assert R1[sv] ** 3 == pytest.approx(R[0] ** 3 + R[1] ** 3, rel=1e-15)
    # total angular momentum (orbital about the origin + spins) is unchanged
    L0 = sum(m[k] * np.cross(x[k], v[k]) + S[k] for k in range(2))
    L1 = M * np.cross(x1[sv], v1[sv]) + S1[sv]
    np.testing.assert_allclose(L1, L0, rtol=1e-13, atol=1e-13 * np.abs(L0).max())
    # kinetic + pair energy before = kinetic of the merged body + Delta U
    E0 = 0.5 * (m[0] * v[0] @ v[0] + m[1] * v[1] @ v[1]) - G * m[0] * m[1] / np.linalg.norm(x[0] - x[1])
    E1 = 0.5 * M * v1[sv] @ v1[sv] + dU
    assert E1 == pytest.approx(E0, rel=1e-13, abs=1e-13 * abs(E0))


@pytest.mark.parametrize("mi,mj,i,j,expect", [(3e-6, 1e-6, 0, 1, 0), (1e-6, 3e-6, 0, 1, 1),
                                              (2e-6, 2e-6, 0, 1, 0), (2e-6, 2e-6, 1, 0, 0)])
def test_survivor_index_rule(mi, mj, i, j, expect):
    """Sec. 7.1: the more massive body survives; equal masses keep the lower index."""
    x, v, m, R, S = _pair(mi=mi, mj=mj)
    assert O.merge(i, j, x, v, m, R, S, G)[6] == expect


def _infall(coll_tol, r0=0.01, Rb=1e-4, mb=1e-3):
    """Two bodies released at rest at separation r0 beside a star of negligible
    mass: radial two-body infall, contact (r = 2 Rb) at the closed-form time
    t(r) = sqrt(r0^3 / 2k) (sqrt(q (1 - q)) + arccos(sqrt q)), q = r/r0, k = G (m_i + m_j).
    (Coordinates of order 0.05 AU: far larger ones would put the 1e-15 error
    control at the resolution of the coordinates.)"""
    x = np.array([[0.05, 0.0, 0.0], [0.05 + r0, 0.0, 0.0]])
    v = np.zeros((2, 3))
    m = np.array([mb, mb])
    R = np.array([Rb, Rb])
    S = np.zeros((2, 3))
    rc = np.array([1e9, 1e9])                  # K = 0: the pair is fully in the BS part
    pairs = np.array([[0, 1]], dtype=np.uint32)
    k = G * 2 * mb
    q = 2 * Rb / r0
    tc = np.sqrt(r0 ** 3 / (2 * k)) * (np.sqrt(q * (1 - q)) + np.arccos(np.sqrt(q)))
    dt = 1.2 * tc
    out = O.bs_groups_coll(x, v, m, R, S, rc[None], pairs, G, 1e-30, dt, coll_tol=coll_tol)
    wc = np.sqrt(2 * k * (1 / (2 * Rb) - 1 / r0))      # approach speed at contact
    return out, tc, wc, x


@pytest.mark.parametrize("coll_tol", [1e-2, 1e-4, 1e-6])
def test_infall_merger_within_collision_precision(coll_tol):
    (x, v, m, R, S, alive, U, log, status, st), tc, wc, x0 = _infall(coll_tol)
    assert status == 0 and len(log) == 1 and list(alive) == [1, 0]
    t, i, j, r, Rs, dU = log[0]
    assert (i, j) == (0, 1)
    overlap = (Rs - r) / Rs
    assert 0.0 < overlap < coll_tol                       # Sec. 7.2 tolerance
    # the merger follows contact within the time the overlap window takes
    assert -1e-9 * tc <= t - tc <= coll_tol * Rs / wc * 1.01 + 1e-9 * tc
    # the survivor stays at the centre of mass, at rest
    np.testing.assert_allclose(x[0], 0.5 * (x0[0] + x0[1]), rtol=1e-14)
    assert np.abs(v[0]).max() < 1e-15 and m[0] == 2e-3 and m[1] == 0.0
    # the pair's energy at release went into U
    assert dU == pytest.approx(-G * 1e-6 / 0.01, rel=1e-9)


def test_without_precision_the_first_overlapping_step_merges():
    (x, v, m, R, S, alive, U, log, status, st), tc, wc, _ = _infall(0.0)
    assert len(log) == 1
    t, i, j, r, Rs, dU = log[0]
    assert t >= tc * (1 - 1e-9) and r < Rs


def test_no_contact_is_the_plain_bulirsch_stoer():
    """Radii too small to touch: the collision path takes the same steps as the
    plain one, bit for bit."""
    wl = disk(160, 0.9, 1.1, 2.0, 31, name="ring-like")
    p = O.make_params(wl)
    x, v, rc, pairs, st = O.step_record(wl.x, wl.v, wl.m, p)
    assert len(pairs) > 0
    xa, va, sa, _ = O.bs_groups(wl.x, wl.v, wl.m, rc[None], pairs, G, wl.m_star, wl.dt)
    R = np.full(wl.n, 1e-12)
    out = O.bs_groups_coll(wl.x, wl.v, wl.m, R, np.zeros((wl.n, 3)), rc[None], pairs, G, wl.m_star,
                           wl.dt, coll_tol=1e-3)
    assert out[8] == sa == 0 and len(out[7]) == 0
    np.testing.assert_array_equal(out[0], xa)
    np.testing.assert_array_equal(out[1], va)


def test_steps_with_mergers_conserve_mass_and_angular_momentum():
    """A dense disk with inflated radii: mergers happen, total mass is unchanged,
    total angular momentum (orbits plus spins) is unchanged to rounding, and the
    bodies merged away carry nothing."""
    wl = disk(160, 0.9, 1.1, 2.0, 31, name="ring-like")
    # radii inflated to R_i + R_j = 6e-3 AU (the critical radii are ~0.04 AU, so pairs
    # meet as encounter pairs first; one pair of the initial disk already overlaps)
    R = np.full(wl.n, 3e-3)
    S = np.zeros((wl.n, 3))
    p = O.make_params(wl, nthreads=4)
    x, v, m, R1, S1, alive, U, log, status, st = O.step_coll(wl.x, wl.v, wl.m, R, S, p, 8,
                                                           coll_tol=1e-3)
    assert status == 0 and len(log) >= 3 and int(alive.sum()) == wl.n - len(log)
    assert m.sum() == pytest.approx(wl.m.sum(), rel=1e-15)
    assert np.all(m[alive == 0] == 0.0) and np.all(R1[alive == 0] == 0.0)
    L0 = (wl.m[:, None] * np.cross(wl.x, wl.v)).sum(axis=0)
    L1 = (m[:, None] * np.cross(x, v)).sum(axis=0) + S1.sum(axis=0)
    np.testing.assert_allclose(L1, L0, rtol=1e-12, atol=1e-12 * np.abs(L0).max())
    # mergers inside a BS call happened at an overlap below the precision (pairs that
    # already overlap when a call starts merge at once, at whatever overlap)
    inside = log[:, 0] > 0.0
    assert inside.any()
    assert np.all((log[inside, 4] - log[inside, 3]) / log[inside, 4] < 1e-3)


def test_mergers_with_two_levels():
    """The same disk under the two-level scheme (Sec. 6.3): the deepest level's BS
    resolves the collisions; mass and angular momentum stay conserved."""
    wl = disk(160, 0.9, 1.1, 2.0, 31, name="ring-like", slevels=2, substeps=10)
    R = np.full(wl.n, 3e-3)
    p = O.make_params(wl, nthreads=4)
    x, v, m, R1, S1, alive, U, log, status, st = O.step_coll(wl.x, wl.v, wl.m, R, np.zeros((wl.n, 3)),
                                                           p, 8, coll_tol=1e-3)
    assert status == 0 and len(log) >= 1 and st["n_pairs"][1] > 0
    assert m.sum() == pytest.approx(wl.m.sum(), rel=1e-15)
    L0 = (wl.m[:, None] * np.cross(wl.x, wl.v)).sum(axis=0)
    L1 = (m[:, None] * np.cross(x, v)).sum(axis=0) + S1.sum(axis=0)
    np.testing.assert_allclose(L1, L0, rtol=1e-12, atol=1e-12 * np.abs(L0).max())
