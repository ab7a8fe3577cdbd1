"""The oracle against the values the paper fixes (tests/golden/paper_values.txt).

Each key of the fixture cites its passage; these tests read the fixture and
check the oracle's changeover function, critical radius, ring grouping and
level factors against it.
"""
import os

import numpy as np
import pytest

import oracle as O
from workloads import ring

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden() -> dict:
    out = {}
    with open(os.path.join(HERE, "golden", "paper_values.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                out[line[0]] = [float(v) for v in line[1:]]
    return out


GOLD = _golden()


def test_changeover_band_edges():
    """Sec. 6.3 footnote: K = 0 for r/rc <= 0.1, 1 for r/rc >= 1, inside (0, 1) between."""
    lo, hi = GOLD["changeover_band"]
    rc = 0.037
    for q in (0.0, 0.03, 0.09999, lo):
        assert O.changeover(q * rc, rc) == 0.0
    for q in (hi, 1.00001, 1.7, 40.0):
        assert O.changeover(q * rc, rc) == 1.0
    for q in np.linspace(lo, hi, 41)[1:-1]:
        assert 0.0 < O.changeover(q * rc, rc) < 1.0


def test_rcrit_constants_define_the_radius():
    """Sec. 2, Eq. rcrit with n1 = 3, n2 = 0.4: rc = max(n1 R_H, n2 dt |v|), checked
    on one body whose Hill term wins and one whose velocity term wins."""
    n1, = GOLD["rcrit_n1"]
    n2, = GOLD["rcrit_n2"]
    x = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    v = np.array([[0.0, 1e-4, 0.0], [0.05, 0.0, 0.0]])
    m = np.array([3e-6, 3e-9])
    dt = 6.0875
    rc = O.rcrit(x, v, m, 1.0, dt, n1, n2)
    hill0 = 1.0 * (3e-6 / 3.0) ** (1.0 / 3.0)
    assert rc[0] == pytest.approx(n1 * hill0, rel=1e-15)
    assert rc[1] == pytest.approx(n2 * dt * 0.05, rel=1e-15)


@pytest.mark.parametrize("n", [6, 12, 15, 16, 40])
def test_ring_partners_and_single_group(n):
    """Sec. 6.2: eight partners per body (all others for N < 16), one group."""
    k, = GOLD["ring_partners"]
    below, = GOLD["ring_all_others_below"]
    wl = ring(n, partners=int(k))
    rc = O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt, wl.n1, wl.n2)
    enc = O.detect(O.precheck(wl.x, rc, wl.f_pc), wl.x, wl.x, rc)
    deg = np.bincount(enc.ravel(), minlength=n)
    assert np.all(deg == (n - 1 if n < below else int(k)))
    assert np.all(O.group(n, enc) == 0)


def _level_factors(r, rcs):
    """The Sec. 6.3 factors for levels with critical radii rcs (level 0 first):
    symplectic level l carries prod_{k<l} (1 - K_k) K_l, Bulirsch-Stoer the rest."""
    out, keep = [], 1.0
    for rc in rcs:
        K = O.changeover(r, rc)
        out.append(keep * K)
        keep *= 1.0 - K
    out.append(keep)
    return out


def test_levels_partition_and_at_most_two_active():
    """Sec. 6.3: with 10 sub-steps per level the velocity term of rc shrinks 10x
    per level, so the changeover bands of neighbouring levels only touch: every
    pair distance is carried by at most two levels, and the factors add to one."""
    sub, = GOLD["levels_substeps"]
    most, = GOLD["levels_max_active"]
    rc0 = 0.02
    rcs = [rc0 / sub ** l for l in range(4)]
    for r in np.geomspace(1e-6 * rc0, 3.0 * rc0, 4001):
        f = _level_factors(r, rcs)
        assert abs(sum(f) - 1.0) <= 4e-16
        assert sum(1 for v in f if v > 0.0) <= most
    # two sub-steps per level (Sec. 6.3 panels c-f): bands overlap, three can be active
    rcs2 = [rc0 / 2 ** l for l in range(4)]
    assert max(sum(1 for v in _level_factors(r, rcs2) if v > 0.0)
               for r in np.geomspace(1e-3 * rc0, rc0, 2001)) > most


def test_semi_active_test_particle_pairs():
    """Sec. 8.1 (TP 2): which pair kinds keep their interaction, read from the
    oracle's kick on four bodies (two large, two test particles) with one body's
    mass switched on at a time."""
    keep_ll, keep_lt, keep_tt = (bool(v) for v in GOLD["tp2_pairs_kept"])
    x = np.array([[1.0, 0.0, 0.0], [1.3, 0.1, 0.0], [0.8, -0.2, 0.1], [1.1, 0.3, -0.1]])
    rc = np.zeros(4)                      # K = 1: plain Newtonian pairs
    nm = 2                                # bodies 0, 1 large; 2, 3 test particles

    def felt(i, j):
        m = np.zeros(4)
        m[j] = 1e-6
        return bool(np.any(O.accel(x, m, rc, 1.0, n_massive=nm)[i] != 0.0))

    assert felt(0, 1) == felt(1, 0) == keep_ll
    assert felt(2, 0) == felt(0, 2) == keep_lt
    assert felt(2, 3) == felt(3, 2) == keep_tt
