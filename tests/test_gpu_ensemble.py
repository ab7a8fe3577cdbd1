"""Batched ensemble with GR and tides (genga_ensemble_*) against the oracle,
system by system, through the C ABI."""
import numpy as np
import pytest

import oracle as O
from workloads.ensemble import Ensemble, ensemble

pytestmark = pytest.mark.gpu


def _oracle_run(wl, s, nsteps, gr=True, tides=True, gr_split=False):
    d = wl.system(s)
    p = O.make_params(G=wl.G, m_star=d["m_star"], dt=d["dt"])
    st = d["star"]
    nn = O.make_nn(gr=gr, tides=tides, c_light=wl.c_light, R_star=st[0], k2_star=st[1],
                   tau_star=st[2], rg2_star=st[3], gr_split=gr_split)
    x, v, w, ws, status, stats = O.step_nn(d["x"], d["v"], d["m"], p, nn, d["R"], d["k2"], d["tau"],
                                           d["rg2"], d["spin"], st[4:7], nsteps)
    assert status == 0
    return x, v, w, ws, stats


def _check(g, ens, wl, systems, nsteps, tol=1e-12, **kw):
    pos = ens.pos.cpu().numpy().T
    vel = ens.vel.cpu().numpy().T
    spin = ens.spin.cpu().numpy().T
    star = ens.star.cpu().numpy()
    worst = 0.0
    for s in systems:
        a, b = wl.offsets[s], wl.offsets[s + 1]
        x, v, w, ws, _ = _oracle_run(wl, s, nsteps, **kw)
        ex = np.max(np.linalg.norm(pos[a:b] - x, axis=1) / np.linalg.norm(x, axis=1))
        ev = np.max(np.linalg.norm(vel[a:b] - v, axis=1) / np.linalg.norm(v, axis=1))
        ew = np.max(np.abs(spin[a:b] - w)) / max(np.abs(w).max(), 1e-300)
        es = np.max(np.abs(star[s, 4:7] - ws)) / np.abs(ws).max()
        worst = max(worst, ex, ev, ew, es)
    assert worst <= tol, worst
    return worst


@pytest.fixture(scope="module")
def small():
    return ensemble(48, seed=123)


def test_ensemble_matches_oracle_gr_and_tides(cuda_lib, small):
    g = cuda_lib
    ens = g.Ensemble(small, g.default_params(G=small.G))
    ens.step(200)
    st = ens.stats()
    assert st["kepler_fail"] == 0 and st["bs_fail"] == 0
    _check(g, ens, small, range(small.n_systems), 200)


@pytest.mark.parametrize("threads,ctas", [(64, 2), (128, 4), (128, 8)])
def test_ensemble_tile_shapes_agree_with_oracle(cuda_lib, small, threads, ctas):
    g = cuda_lib
    ens = g.Ensemble(small, g.default_params(G=small.G))
    ens.set_tile(threads, ctas)
    ens.step(50)
    _check(g, ens, small, range(0, small.n_systems, 5), 50)


def test_ensemble_thirty_two_threads_for_small_systems(cuda_lib):
    g = cuda_lib
    wl = ensemble(40, seed=7, nmin=1, nmax=32)
    ens = g.Ensemble(wl, g.default_params(G=wl.G))
    ens.set_tile(32, 8)
    ens.step(60)
    _check(g, ens, wl, range(wl.n_systems), 60)


def test_ensemble_gr_only_and_tides_only(cuda_lib, small):
    g = cuda_lib
    for gr, tides in ((True, False), (False, True)):
        ens = g.Ensemble(small, g.default_params(G=small.G), gr=gr, tides=tides)
        ens.step(40)
        _check(g, ens, small, range(0, small.n_systems, 7), 40, gr=gr, tides=tides)


def test_ensemble_graph_replay_is_deterministic(cuda_lib, small):
    g = cuda_lib
    a = g.Ensemble(small, g.default_params(G=small.G))
    a.step(10)
    a.step(10)
    b = g.Ensemble(small, g.default_params(G=small.G))
    b.step(20)
    assert np.array_equal(a.pos.cpu().numpy(), b.pos.cpu().numpy())
    assert np.array_equal(a.spin.cpu().numpy(), b.spin.cpu().numpy())


def test_ensemble_autotune_restores_state(cuda_lib, small):
    g = cuda_lib
    ens = g.Ensemble(small, g.default_params(G=small.G))
    before = (ens.pos.clone(), ens.vel.clone(), ens.spin.clone(), ens.star.clone())
    threads, ctas = ens.autotune(5)
    assert threads in (64, 128) and ctas in (2, 4, 8)
    for t0, t1 in zip(before, (ens.pos, ens.vel, ens.spin, ens.star)):
        assert bool((t0 == t1).all())


def test_ensemble_close_encounter_inside_a_system(cuda_lib):
    """Two planets of one system start inside each other's critical radius:
    the in-CTA detection, grouping and Bulirsch-Stoer run and match the oracle."""
    g = cuda_lib
    wl = ensemble(6, seed=99, nmin=8, nmax=12)
    # planet 1 of every system 4% outside planet 0 in the same direction, on a
    # circular orbit: about 1.5 mutual Hill radii apart, inside r_crit
    for s in range(wl.n_systems):
        a = wl.offsets[s]
        x1 = wl.x[a] * 1.04
        wl.x[a + 1] = x1
        vc = np.sqrt(wl.G * (wl.m_star[s] + wl.m[a + 1]) / np.linalg.norm(x1))
        wl.v[a + 1] = vc * np.cross([0.0, 0.0, 1.0], x1 / np.linalg.norm(x1))
    ens = g.Ensemble(wl, g.default_params(G=wl.G))
    ens.step(30)
    st = ens.stats()
    assert st["n_pairs"][0] > 0 and st["n_groups"] > 0
    _check(g, ens, wl, range(wl.n_systems), 30, tol=1e-11)


def test_ensemble_angular_momentum_report_matches_oracle(cuda_lib, small):
    g = cuda_lib
    ens = g.Ensemble(small, g.default_params(G=small.G), gr=False, tides=True)
    L = ens.angmom()
    for s in range(0, small.n_systems, 11):
        d = small.system(s)
        Lr = O.angmom_spin(d["x"], d["v"], d["m"], d["R"], d["rg2"], d["spin"], d["m_star"],
                           d["star"][0], d["star"][3], d["star"][4:7])
        np.testing.assert_allclose(L[s], Lr, rtol=1e-13, atol=1e-30)


def test_ensemble_mixed_kick_matches_oracle(cuda_lib, small):
    """The mixed-precision pair kick in the ensemble (FP64 displacement and
    accumulation, float-float r^-3): 200 steps of 48 systems with GR and tides
    against the FP64 oracle within the mixed form's bound (1e-9), with the
    pre-check candidates and encounter counts of the FP64 form."""
    g = cuda_lib
    mixed = g.Ensemble(small, g.default_params(G=small.G, precision=g.GENGA_MIXED))
    mixed.step(200)
    fp64 = g.Ensemble(small, g.default_params(G=small.G))
    fp64.step(200)
    sm, sf = mixed.stats(), fp64.stats()
    assert sm["kepler_fail"] == 0 and sm["bs_fail"] == 0
    assert sm["n_candidates"] == sf["n_candidates"] and sm["n_pairs"][0] == sf["n_pairs"][0]
    _check(g, mixed, small, range(small.n_systems), 200, tol=1e-9)


def test_ensemble_mixed_close_encounter(cuda_lib):
    """Mixed kick with encounters inside the systems: the candidates and pairs
    equal the FP64 form's and the states stay within the mixed bound."""
    g = cuda_lib
    wl = ensemble(6, seed=99, nmin=8, nmax=12)
    for s in range(wl.n_systems):
        a = wl.offsets[s]
        x1 = wl.x[a] * 1.04
        wl.x[a + 1] = x1
        vc = np.sqrt(wl.G * (wl.m_star[s] + wl.m[a + 1]) / np.linalg.norm(x1))
        wl.v[a + 1] = vc * np.cross([0.0, 0.0, 1.0], x1 / np.linalg.norm(x1))
    mixed = g.Ensemble(wl, g.default_params(G=wl.G, precision=g.GENGA_MIXED))
    mixed.step(30)
    fp64 = g.Ensemble(wl, g.default_params(G=wl.G))
    fp64.step(30)
    sm, sf = mixed.stats(), fp64.stats()
    assert sm["n_pairs"][0] > 0 and sm["n_pairs"][0] == sf["n_pairs"][0]
    assert sm["n_candidates"] == sf["n_candidates"]
    _check(g, mixed, wl, range(wl.n_systems), 30, tol=1e-9)


@pytest.mark.parametrize("tides", [True, False])
def test_ensemble_gr_split_matches_oracle(cuda_lib, small, tides):
    """GR by the Hamiltonian splitting of Sec. 3.1 (pseudovelocities between the
    conversions, alpha-scaled drift, sun kick, gamma term with HC), with and
    without tides: 200 steps of 48 systems against the oracle."""
    g = cuda_lib
    ens = g.Ensemble(small, g.default_params(G=small.G), tides=tides, gr_split=True)
    ens.step(200)
    st = ens.stats()
    assert st["kepler_fail"] == 0 and st["bs_fail"] == 0
    _check(g, ens, small, range(small.n_systems), 200, tides=tides, gr_split=True)


def test_ensemble_gr_split_close_encounter(cuda_lib):
    """Splitting with encounters: the Bulirsch-Stoer groups run with the alpha
    factor on each member's Kepler terms; against the oracle."""
    g = cuda_lib
    wl = ensemble(6, seed=99, nmin=8, nmax=12)
    for s in range(wl.n_systems):
        a = wl.offsets[s]
        x1 = wl.x[a] * 1.04
        wl.x[a + 1] = x1
        vc = np.sqrt(wl.G * (wl.m_star[s] + wl.m[a + 1]) / np.linalg.norm(x1))
        wl.v[a + 1] = vc * np.cross([0.0, 0.0, 1.0], x1 / np.linalg.norm(x1))
    ens = g.Ensemble(wl, g.default_params(G=wl.G), gr_split=True)
    ens.step(30)
    assert ens.stats()["n_groups"] > 0
    _check(g, ens, wl, range(wl.n_systems), 30, tol=1e-11, gr_split=True)
