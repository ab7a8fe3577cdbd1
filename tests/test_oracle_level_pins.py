"""Pins of the oracle's higher-level changeover scheme (Sec. 6.3, Appendix A
SEnc) by what the mathematics fixes:

* the level split of a pair force: the level-0 Kick carries K_0, KickS at
  level l carries prod_{k<l} (1 - K_k) K_l, the deepest level's
  Bulirsch-Stoer derivative carries prod_k (1 - K_k); the factors telescope to
  1, so the parts the oracle's own routines produce (orc_level_force_parts:
  its all-pairs kick, its KickS routine and its Bulirsch-Stoer derivative) must
  add up to the plain Newtonian pair force at every separation, across every
  band of every level;
* the whole multi-level step is a second-order integrator of the exact
  dynamics: against a DOP853 integration of the democratic-heliocentric
  equations (the same reference as the one-level convergence pin) the error
  falls by ~4x per halving of dt when a close pair goes through the
  changeover bands of both levels.  A wrong factor product integrates another
  Hamiltonian, and a wrong restart state of the level bodies breaks
  consistency; both stall the convergence.
"""
import numpy as np
import pytest

import oracle as O
from tests.test_oracle_pins import _few_body, _reference_dhc
from workloads import G_GAUSS as G


def _newton(x, m):
    n = len(m)
    a = np.zeros((n, 3))
    for i in range(n):
        for j in range(n):
            if i != j:
                d = x[j] - x[i]
                r = np.sqrt(d @ d)
                a[i] += G * m[j] * d / r**3
    return a


def _all_pairs(n):
    return np.array([(i, j) for i in range(n) for j in range(i + 1, n)], dtype=np.uint32)


@pytest.mark.parametrize("rc_levels", [(0.03, 0.01), (0.03, 0.012, 0.004), (0.02, 0.02)])
def test_level_parts_sum_to_newton_across_every_band(rc_levels):
    """Two bodies swept from well inside the deepest level's inner radius to
    beyond rc_0: kick + KickS parts + BS part = Newtonian force, to rounding."""
    nlev = len(rc_levels)
    m = np.array([3e-6, 7e-6])
    rs = np.geomspace(0.05 * min(rc_levels), 1.3 * max(rc_levels), 400)
    in_band = np.zeros(nlev, dtype=int)
    u = np.array([0.48, -0.6, 0.64])
    u /= np.linalg.norm(u)
    for r in rs:
        x = np.array([[1.0, 0.2, -0.1], [1.0, 0.2, -0.1]])
        x[1] += r * u
        rcl = np.array([[rc, rc] for rc in rc_levels])
        ak, aks, ab = O.level_force_parts(x, m, rcl, _all_pairs(2), G)
        total = ak + aks.sum(axis=0) + ab
        ref = _newton(x, m)
        assert np.abs(total - ref).max() <= 2e-15 * np.abs(ref).max(), (r, total, ref)
        # the parts are each a fraction in [0, 1] of the force, along it
        for part in [ak, *aks, ab]:
            w = (part[0] @ ref[0]) / (ref[0] @ ref[0])
            assert -1e-15 <= w <= 1 + 1e-15
        for level, rc in enumerate(rc_levels):
            in_band[level] += 0.1 * rc < r < rc
    assert (in_band > 10).all()          # every band was crossed


def test_level_parts_outside_the_bands_are_exact():
    """Beyond rc_0 the whole force is the level-0 kick's; inside 0.1 rc of every
    level it is all Bulirsch-Stoer's; between the levels' bands all of it sits
    on the one KickS level whose band lies outside r."""
    m = np.array([2e-6, 5e-6])
    rc_levels = (0.05, 0.004)
    rcl = np.array([[rc, rc] for rc in rc_levels])
    for r, who in [(0.06, "kick"), (0.0003, "bs"), (0.0045, "kickS")]:
        x = np.array([[0.7, -0.3, 0.0], [0.7, -0.3, 0.0]])
        x[1, 0] += r
        ak, aks, ab = O.level_force_parts(x, m, rcl, _all_pairs(2), G)
        ref = _newton(x, m)
        parts = {"kick": ak, "kickS": aks[0], "bs": ab}
        if who == "kickS":
            # r = 0.0045 is inside rc_0's inner radius 0.005 (K_0 = 0) and
            # beyond rc_1 (K_1 = 1): KickS takes (1 - 0) * 1 of the force
            assert np.array_equal(parts["kick"], np.zeros_like(ak))
            assert np.abs(parts["bs"]).max() == 0.0
        for name, part in parts.items():
            if name == who:
                assert np.abs(part - ref).max() <= 2e-16 * np.abs(ref).max()
            else:
                assert np.abs(part).max() == 0.0, name


def test_level_parts_many_bodies():
    """A 6-body cluster whose pairs span every band: the parts of every body
    sum to its Newtonian pair acceleration."""
    rng = np.random.default_rng(5)
    # pairs at three scales: far apart, inside rc_0, inside the deepest radius
    x = np.array([1.0, 0.0, 0.0]) + 0.02 * rng.standard_normal((6, 3))
    x[1] = x[0] + 0.004 * rng.standard_normal(3)
    x[2] = x[0] + 0.0004 * rng.standard_normal(3)
    x[4] = x[3] + 0.001 * rng.standard_normal(3)
    m = rng.uniform(1e-6, 9e-6, 6)
    rc0 = rng.uniform(0.01, 0.04, 6)
    rcl = np.array([rc0, 0.3 * rc0, 0.08 * rc0])
    ak, aks, ab = O.level_force_parts(x, m, rcl, _all_pairs(6), G)
    ref = _newton(x, m)
    total = ak + aks.sum(axis=0) + ab
    assert np.abs(total - ref).max() <= 2e-15 * np.abs(ref).max()
    assert np.abs(aks).max() > 0 and np.abs(ab).max() > 0 and np.abs(ak).max() > 0


@pytest.mark.parametrize("slevels,substeps", [(2, 10), (3, 2)])
def test_multilevel_step_second_order_convergence(slevels, substeps):
    """Multi-level steps on the close few-body system: errors against the exact
    dynamics fall ~4x per halving of dt (the Hill-only critical radius keeps
    the split fixed as dt shrinks), and the higher levels do run."""
    x, v, m = _few_body(close=True)
    T = 96.0
    xr, _ = _reference_dhc(x, v, m, 1.0, T)
    errs = []
    for nst in [16, 32, 64]:
        p = O.make_params(dt=T / nst, n1=3.0, n2=0.0, f_pc=4.0, slevels=slevels, substeps=substeps)
        x1, _, st, stats = O.step(x, v, m, p, nst)
        assert st == 0
        assert stats["n_pairs"][slevels - 1] > 0 and stats["n_groups"] > 0
        errs.append(np.abs(x1 - xr).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, errs
