"""Pins of the oracle's semi-active test-particle mode (Sec. 8.1, TP 2; reading R24).

A test particle (index >= n_massive) has no interaction with another test
particle and interacts with the large bodies as in the fully interactive mode.
Each test reaches the expected value by a route that does not use the masking
itself: removing the other test particles from the system, filtering the full
candidate list, a brute-force sum of the dropped potential terms, or the
interaction-free composition of HC and Kepler drifts.
"""
import numpy as np
import pytest

import oracle as O
from workloads import G_GAUSS, config_workload, disk

G = G_GAUSS


def _small(n=90, seed=31):
    wl = disk(n, 0.5, 0.8, 2.0, seed, name="tp")
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    return wl, rc


def test_test_particle_feels_only_large_bodies():
    """Row i of a test particle equals row i of the system made of the large bodies
    and i alone (same sources in the same order: bit for bit); rows of large
    bodies equal the fully interactive rows."""
    wl, rc = _small()
    nm = 55
    a_tp = O.accel(wl.x, wl.m, rc, G, n_massive=nm)
    a_full = O.accel(wl.x, wl.m, rc, G)
    np.testing.assert_array_equal(a_tp[:nm], a_full[:nm])
    for i in (nm, nm + 7, wl.n - 1):
        keep = np.r_[np.arange(nm), i]
        a_sub = O.accel(wl.x[keep], wl.m[keep], rc[keep], G)
        np.testing.assert_array_equal(a_tp[i], a_sub[-1])
    assert np.any(a_tp[nm:] != a_full[nm:])      # the test-particle pairs did act before


def test_semi_active_kick_conserves_momentum():
    """Large bodies still feel the test particles (semi-active): pair forces stay
    symmetric, so sum_i m_i a_i vanishes."""
    wl, rc = _small()
    a = O.accel(wl.x, wl.m, rc, G, n_massive=40)
    F = wl.m[:, None] * a
    assert np.abs(F.sum(axis=0)).max() < 1e-13 * np.abs(F).sum(axis=0).max()


@pytest.mark.parametrize("nm", [0, 1, 45, 89, 90])
def test_candidates_are_the_full_list_without_test_particle_pairs(nm):
    wl, rc = _small()
    full = O.precheck(wl.x, rc, wl.f_pc)
    keep = full[(full[:, 0] < nm) | (full[:, 1] < nm)]
    np.testing.assert_array_equal(O.precheck(wl.x, rc, wl.f_pc, n_massive=nm), keep)


def test_energy_drops_exactly_the_test_particle_pair_terms():
    wl, _ = _small()
    nm = 50
    E_full, L_full = O.energy(wl.x, wl.v, wl.m, wl.m_star, G)
    E_tp, L_tp = O.energy(wl.x, wl.v, wl.m, wl.m_star, G, n_massive=nm)
    dropped = 0.0
    for i in range(nm, wl.n):
        for j in range(i + 1, wl.n):
            dropped += G * wl.m[i] * wl.m[j] / np.linalg.norm(wl.x[j] - wl.x[i])
    assert abs((E_tp - E_full) - dropped) <= 1e-13 * abs(E_full)
    np.testing.assert_array_equal(L_tp, L_full)


def test_only_test_particles_step_is_hc_and_kepler():
    """n_massive = 0: no pair interacts, so a step is HC(dt/2), Kepler drift, HC(dt/2)."""
    wl = config_workload(0, n_override=64)
    p = O.make_params(wl, tp_mode=2, n_massive=0)
    x, v, status, st = O.step(wl.x, wl.v, wl.m, p, 1)
    assert status == 0 and st["n_candidates"] == 0 and st["n_pairs"][0] == 0
    x1 = O.hc(wl.x, wl.v, wl.m, wl.m_star, 0.5 * wl.dt)
    x2, v2, fails = O.drift(x1, wl.v, G * wl.m_star, wl.dt)
    x3 = O.hc(x2, v2, wl.m, wl.m_star, 0.5 * wl.dt)
    np.testing.assert_array_equal(x, x3)
    np.testing.assert_array_equal(v, v2)


def test_no_test_particles_is_the_fully_interactive_step():
    wl = config_workload(0, n_override=256)
    xa, va, sa, _ = O.step(wl.x, wl.v, wl.m, O.make_params(wl), 2)
    xb, vb, sb, _ = O.step(wl.x, wl.v, wl.m, O.make_params(wl, tp_mode=2, n_massive=wl.n), 2)
    assert sa == sb == 0
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
