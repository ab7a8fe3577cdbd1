"""Pins of the oracle's GR (Sec. 3, Eq. apn) and tidal (Sec. 4.1-4.2) forces,
applied by the implicit midpoint rule (Sec. 2.3), against closed forms:
  * GR: the perihelion advance per orbit 6 pi G M / (c^2 a (1 - e^2));
  * tides: the secular da/dt of a circular orbit implied by the transverse
    tidal force, da/dt = 2 F_theta / (m n) with
    F_theta = P_i (W_i - n) + P_s (W_s - n), P = 3 G m_1^2 R^5 k2 tau / a^7;
  * tides: total angular momentum (orbit + planet spin + star spin) of a
    one-planet system is conserved.
"""
import numpy as np
import pytest

import oracle as O
from tests import twobody
from workloads import G_GAUSS

G = G_GAUSS
C_LIGHT = 173.1446326846693


def _elements(x, v, mu):
    E, h, A = twobody.invariants(x, v, mu)
    a = float(-mu / (2 * E))
    e = float(np.linalg.norm(A.astype(float)) / mu)
    varpi = float(np.arctan2(float(A[1]), float(A[0])))
    return a, e, varpi


def _one_planet(a, e, m, m_star=1.0):
    mu = G * (m_star + m)
    r = a * (1 - e)
    vp = np.sqrt(mu * (1 + e) / r)
    x = np.array([[r, 0.0, 0.0]])
    vh = np.array([[0.0, vp, 0.0]])
    vb = vh - m * vh / (m_star + m)
    return x, vb, np.array([m])


def test_gr_perihelion_advance_matches_closed_form():
    a, e, m = 0.05, 0.2, 1e-9
    x, v, mm = _one_planet(a, e, m)
    mu = G * (1 + m)
    P = 2 * np.pi * np.sqrt(a ** 3 / mu)
    norb, per = 50, 400
    p = O.make_params(G=G, m_star=1.0, dt=P / per, n1=0.0, n2=0.0)
    nn = O.make_nn(gr=True, tides=False)
    z = np.zeros(1)
    spin = np.zeros((1, 3))
    x1, v1, *_ = O.step_nn(x, v, mm, p, nn, z, z, z, z, spin, np.zeros(3), norb * per)
    u0 = v[0] + m * v[0] / 1.0          # heliocentric velocity
    u1 = v1[0] + m * v1[0] / 1.0
    _, _, w0 = _elements(x[0], u0, mu)
    _, _, w1 = _elements(x1[0], u1, mu)
    measured = (w1 - w0) / norb
    expected = 6 * np.pi * mu / (C_LIGHT ** 2 * a * (1 - e * e))
    assert abs(measured / expected - 1) < 0.01, (measured, expected)


def _tidal_setup(W_planet):
    a, m, m_star = 0.02, 3e-6, 1.0
    x, v, mm = _one_planet(a, 0.0, m, m_star)
    R = np.array([1e-4])
    k2 = np.array([0.3])
    tau = np.array([1e-5])
    rg2 = np.array([0.33])
    spin = np.array([[0.0, 0.0, W_planet]])
    star = dict(R_star=0.005, k2_star=0.03, tau_star=2e-6, rg2_star=0.07)
    spin_star = np.array([0.0, 0.0, 0.5])
    return a, m, m_star, x, v, mm, R, k2, tau, rg2, spin, star, spin_star


@pytest.mark.parametrize("W_planet", [30.0, 1.0])
def test_tidal_da_dt_matches_closed_form(W_planet):
    a, m, m_star, x, v, mm, R, k2, tau, rg2, spin, star, spin_star = _tidal_setup(W_planet)
    mu = G * (m_star + m)
    n = np.sqrt(mu / a ** 3)
    P = 2 * np.pi / n
    nst, per = 4, 200
    p = O.make_params(G=G, m_star=m_star, dt=P / per, n1=0.0, n2=0.0)
    nn = O.make_nn(gr=False, tides=True, **star)
    x1, v1, spin1, ss1, st, _ = O.step_nn(x, v, mm, p, nn, R, k2, tau, rg2, spin, spin_star,
                                          nst * per)
    assert st == 0
    u0 = v[0] * (1 + m / m_star)
    u1 = v1[0] * (1 + m / m_star)
    # osculating a with the conservative tidal radial term removed: use the
    # orbit-averaged change of the specific angular momentum instead,
    # h = sqrt(mu a) for a circular orbit -> da/dt = 2 sqrt(a/mu) dh/dt
    h0 = np.linalg.norm(np.cross(x[0], u0))
    h1 = np.linalg.norm(np.cross(x1[0], u1))
    T = nst * P
    dadt_measured = 2 * np.sqrt(a / mu) * (h1 - h0) / T
    Wp = 0.5 * (spin[0, 2] + spin1[0, 2])
    Ws = 0.5 * (spin_star[2] + ss1[2])
    Pi = 3 * G * m_star ** 2 * R[0] ** 5 * k2[0] * tau[0] / a ** 7
    Ps = 3 * G * m ** 2 * star["R_star"] ** 5 * star["k2_star"] * star["tau_star"] / a ** 7
    F_theta = Pi * (Wp - n) + Ps * (Ws - n)
    dadt_expected = 2 * F_theta / (m * n)
    assert np.sign(dadt_measured) == np.sign(W_planet - n)
    assert abs(dadt_measured / dadt_expected - 1) < 0.02, (dadt_measured, dadt_expected)


def test_tides_conserve_total_angular_momentum_one_planet():
    a, m, m_star, x, v, mm, R, k2, tau, rg2, spin, star, spin_star = _tidal_setup(30.0)
    tau = tau * 100.0                                  # strong dissipation
    xe, ve, _ = _one_planet(a, 0.1, m, m_star)
    p = O.make_params(G=G, m_star=m_star, dt=0.01, n1=0.0, n2=0.0)
    nn = O.make_nn(gr=False, tides=True, **star)
    L0 = O.angmom_spin(xe, ve, mm, R, rg2, spin, m_star, star["R_star"], star["rg2_star"], spin_star)
    x1, v1, spin1, ss1, st, _ = O.step_nn(xe, ve, mm, p, nn, R, k2, tau, rg2, spin, spin_star, 2000)
    L1 = O.angmom_spin(x1, v1, mm, R, rg2, spin1, m_star, star["R_star"], star["rg2_star"], ss1)
    Lorb0 = np.linalg.norm(mm[0] * np.cross(xe[0], ve[0]))
    Lorb1 = np.linalg.norm(mm[0] * np.cross(x1[0], v1[0]))
    assert abs(Lorb1 - Lorb0) > 1e-6 * Lorb0          # the orbit really exchanges L with spins
    assert np.abs(L1 - L0).max() < 1e-12 * np.linalg.norm(L0)


def test_nn_off_reduces_to_plain_step():
    a, m, m_star, x, v, mm, R, k2, tau, rg2, spin, star, spin_star = _tidal_setup(30.0)
    p = O.make_params(G=G, m_star=m_star, dt=0.01, n1=0.0, n2=0.0)
    nn = O.make_nn(gr=False, tides=False, **star)
    x1, v1, *_ = O.step_nn(x, v, mm, p, nn, R, k2, tau, rg2, spin, spin_star, 50)
    x2, v2, *_ = O.step(x, v, mm, p, 50)
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(v1, v2)


# ---------------------------------------------------------------- GR splitting (Sec. 3.1)
def _h1pn(x, v, mu):
    """The standard first post-Newtonian two-body Hamiltonian per unit mass of a
    test particle, H = u^2/2 - mu/r - u^4/(8c^2) - 3 mu u^2/(2 c^2 r) + mu^2/(2 c^2 r^2),
    with the canonical velocity u taken from the real one through that
    Hamiltonian's own dx/dt = dH/du = u (1 - u^2/(2c^2) - 3 mu/(c^2 r))."""
    c2 = C_LIGHT ** 2
    r = np.linalg.norm(x)
    u = v.copy()
    for _ in range(4):
        u2 = u @ u
        u = v / (1 - u2 / (2 * c2) - 3 * mu / (c2 * r))
    u2 = u @ u
    return u2 / 2 - mu / r - u2 * u2 / (8 * c2) - 3 * mu * u2 / (2 * c2 * r) + mu * mu / (2 * c2 * r * r)


def test_gr_split_perihelion_advance_matches_closed_form():
    """The Hamiltonian splitting of Sec. 3.1 gives the same perihelion advance per
    orbit as the closed form 6 pi G M / (c^2 a (1 - e^2))."""
    a, e, m = 0.05, 0.2, 1e-9
    x, v, mm = _one_planet(a, e, m)
    mu = G * (1 + m)
    P = 2 * np.pi * np.sqrt(a ** 3 / mu)
    norb, per = 50, 400
    p = O.make_params(G=G, m_star=1.0, dt=P / per, n1=0.0, n2=0.0)
    nn = O.make_nn(gr=True, tides=False, gr_split=True)
    z = np.zeros(1)
    x1, v1, *_ = O.step_nn(x, v, mm, p, nn, z, z, z, z, np.zeros((1, 3)), np.zeros(3), norb * per)
    _, _, w0 = _elements(x[0], v[0] + m * v[0], mu)
    _, _, w1 = _elements(x1[0], v1[0] + m * v1[0], mu)
    measured = (w1 - w0) / norb
    expected = 6 * np.pi * mu / (C_LIGHT ** 2 * a * (1 - e * e))
    assert abs(measured / expected - 1) < 0.01, (measured, expected)


def test_gr_split_conserves_the_first_post_newtonian_energy():
    """The split step is a symplectic map of the 1PN Hamiltonian: that energy
    stays within the small splitting oscillation over 20 orbits, while the
    Newtonian energy of the same orbit swings by far more (the PN terms exchange
    energy with it along the orbit).  A wrong sign or factor in any of the
    alpha, beta, gamma terms integrates another Hamiltonian and fails this."""
    a, e, m = 0.05, 0.4, 1e-12
    x, v, mm = _one_planet(a, e, m)
    mu = G * (1 + m)
    P = 2 * np.pi * np.sqrt(a ** 3 / mu)
    per = 800
    p = O.make_params(G=G, m_star=1.0, dt=P / per, n1=0.0, n2=0.0)
    nn = O.make_nn(gr=True, tides=False, gr_split=True)
    z = np.zeros(1)
    H0 = _h1pn(x[0], v[0], mu)
    EN0 = 0.5 * v[0] @ v[0] - mu / np.linalg.norm(x[0])
    dH, dEN = [], []
    xs, vs = x, v
    for _ in range(40):                      # 20 orbits in half-orbit chunks
        xs, vs, *_ = O.step_nn(xs, vs, mm, p, nn, z, z, z, z, np.zeros((1, 3)), np.zeros(3), per // 2)
        dH.append(abs(_h1pn(xs[0], vs[0], mu) - H0) / abs(H0))
        dEN.append(abs(0.5 * vs[0] @ vs[0] - mu / np.linalg.norm(xs[0]) - EN0) / abs(EN0))
    assert max(dH) < 2e-10, max(dH)
    assert max(dEN) > 50 * max(dH), (max(dEN), max(dH))


def test_gr_split_real_and_pseudo_velocities():
    """With c so large that 1/c^2 vanishes, the split step is the plain step bit
    for bit (every GR term, the velocity conversions and the drift-time factor
    reduce to the identity); the implicit and split forms of GR agree on a
    several-planet system to the size of the 1PN terms times the step's error."""
    from workloads.ensemble import ensemble
    wl = ensemble(3, seed=5)
    d = wl.system(0)
    p = O.make_params(G=wl.G, m_star=d["m_star"], dt=d["dt"])
    z = np.zeros(len(d["m"]))
    args = (d["R"], d["k2"], d["tau"], d["rg2"], np.zeros((len(d["m"]), 3)), np.zeros(3))
    plain = O.step_nn(d["x"], d["v"], d["m"], p, O.make_nn(gr=False, tides=False), *args, 50)
    huge = O.step_nn(d["x"], d["v"], d["m"], p, O.make_nn(gr=True, tides=False, gr_split=True,
                                                          c_light=1e300), *args, 50)
    np.testing.assert_array_equal(huge[0], plain[0])
    np.testing.assert_array_equal(huge[1], plain[1])
    imp = O.step_nn(d["x"], d["v"], d["m"], p, O.make_nn(gr=True, tides=False), *args, 50)
    spl = O.step_nn(d["x"], d["v"], d["m"], p, O.make_nn(gr=True, tides=False, gr_split=True), *args, 50)
    gr_shift = np.abs(imp[0] - plain[0]).max()
    assert gr_shift > 0
    assert np.abs(spl[0] - imp[0]).max() < 0.05 * gr_shift
