"""Pins of the oracle's frozen-encounter step and its tangent-linear
derivative (the adjoint configuration): the recorded step equals the normal
step bit for bit, replaying the recorded rc and pairs reproduces it, and the
tangent agrees with central finite differences taken with the same frozen
lists; the tangent is linear in the perturbation."""
import numpy as np
import pytest

import oracle as O
from workloads import config_workload, disk


def _run(wl, nsteps):
    p = O.make_params(wl, nthreads=4)
    x, v = wl.x, wl.v
    rec = []
    for _ in range(nsteps):
        x, v, rc, pairs, st = O.step_record(x, v, wl.m, p)
        assert st == 0
        rec.append((rc, pairs))
    return x, v, rec, p


def _replay(x, v, m, p, rec, dx=None, dv=None, dm=None):
    for rc, pairs in rec:
        x, v, dx, dv, st = O.step_frozen(x, v, m, p, rc, pairs, dx, dv, dm)
        assert st == 0
    return x, v, dx, dv


@pytest.fixture(scope="module")
def dense():
    # dense enough for encounter groups in a few steps
    return disk(160, 0.9, 1.1, 2.0, 31, name="ring-like")


def test_recorded_and_frozen_steps_equal_normal_step(dense):
    wl = dense
    x, v, rec, p = _run(wl, 6)
    xr, vr, st, stats = O.step(wl.x, wl.v, wl.m, p, 6)
    assert stats["n_pairs"][0] > 0
    np.testing.assert_array_equal(x, xr)
    np.testing.assert_array_equal(v, vr)
    xf, vf, _, _ = _replay(wl.x, wl.v, wl.m, p, rec)
    np.testing.assert_array_equal(xf, xr)
    np.testing.assert_array_equal(vf, vr)


def test_tangent_matches_central_differences(dense):
    wl = dense
    x1, v1, rec, p = _run(wl, 6)
    assert sum(len(r[1]) for r in rec) > 0
    rng = np.random.default_rng(3)
    # direction in state units (AU, AU/day, mass): central differences with a
    # step of h = 1e-7 of those units
    dx0 = rng.standard_normal(wl.x.shape)
    dv0 = rng.standard_normal(wl.v.shape) * 0.017
    dm0 = rng.standard_normal(wl.m.shape) * wl.m
    _, _, dx, dv = _replay(wl.x, wl.v, wl.m, p, rec, dx0, dv0, dm0)
    eps = 1e-7
    xp, vp, _, _ = _replay(wl.x + eps * dx0, wl.v + eps * dv0, wl.m + eps * dm0, p, rec)
    xm, vm, _, _ = _replay(wl.x - eps * dx0, wl.v - eps * dv0, wl.m - eps * dm0, p, rec)
    fdx = (xp - xm) / (2 * eps)
    fdv = (vp - vm) / (2 * eps)
    assert np.abs(fdx - dx).max() <= 1e-6 * np.abs(dx).max()
    assert np.abs(fdv - dv).max() <= 1e-6 * np.abs(dv).max()


def test_tangent_is_linear(dense):
    wl = dense
    _, _, rec, p = _run(wl, 3)
    rng = np.random.default_rng(4)
    a = [rng.standard_normal(wl.x.shape) * 1e-3, rng.standard_normal(wl.v.shape) * 1e-5,
         rng.standard_normal(wl.m.shape) * wl.m]
    b = [rng.standard_normal(wl.x.shape) * 1e-3, rng.standard_normal(wl.v.shape) * 1e-5,
         rng.standard_normal(wl.m.shape) * wl.m]
    _, _, ax, av = _replay(wl.x, wl.v, wl.m, p, rec, *a)
    _, _, bx, bv = _replay(wl.x, wl.v, wl.m, p, rec, *b)
    s = [ai + 2 * bi for ai, bi in zip(a, b)]
    _, _, sx, sv = _replay(wl.x, wl.v, wl.m, p, rec, *s)
    np.testing.assert_allclose(sx, ax + 2 * bx, rtol=0, atol=1e-11 * np.abs(sx).max())
    np.testing.assert_allclose(sv, av + 2 * bv, rtol=0, atol=1e-11 * np.abs(sv).max())


def test_frozen_tangent_matches_the_free_step(dense):
    """The derivative with frozen rc and pairs is the derivative of the normal
    step (rc recomputed, encounters detected anew) as long as the perturbation
    changes no encounter decision: central differences of 6 normal steps agree
    with the tangent of the frozen replay."""
    wl = dense
    _, _, rec, p = _run(wl, 6)
    rng = np.random.default_rng(1)
    dx0 = rng.standard_normal(wl.x.shape) * 1e-3
    dv0 = rng.standard_normal(wl.v.shape) * 1e-5
    dm0 = np.zeros(wl.n)
    w = rng.standard_normal(wl.x.shape)
    _, _, dx, _ = _replay(wl.x, wl.v, wl.m, p, rec, dx0, dv0, dm0)
    h = 1e-5
    xp, _, sp, stp = O.step(wl.x + h * dx0, wl.v + h * dv0, wl.m, p, 6)
    xm, _, sm, stm = O.step(wl.x - h * dx0, wl.v - h * dv0, wl.m, p, 6)
    assert sp == sm == 0
    # the perturbed runs find the same encounters as the recording
    assert stp["n_pairs"][0] == stm["n_pairs"][0] == sum(len(r[1]) for r in rec)
    tangent = float((w * dx).sum())
    fd = float((w * (xp - xm)).sum()) / (2 * h)
    assert abs(fd - tangent) <= 1e-6 * abs(tangent)
