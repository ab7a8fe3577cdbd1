"""Exact two-body propagation by the classical anomaly route (test helper).

Independent of the universal-variable drift under test: it converts the state
to orbital elements, advances the mean anomaly, solves Kepler's equation by
bisection in extended precision and rebuilds the state with the Gauss f and g
functions written in the eccentric (or hyperbolic) anomaly difference.
"""
import numpy as np

LD = np.longdouble


def _bisect(fun, lo, hi, iters=200):
    flo = fun(lo)
    for _ in range(iters):
        mid = (lo + hi) / 2
        fm = fun(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
        if hi - lo <= abs(mid) * LD(1e-19) + LD(1e-300):
            break
    return (lo + hi) / 2


def propagate(x0, v0, mu, dt):
    """State after time dt on the Kepler orbit about mu (elliptic or hyperbolic)."""
    x0 = np.asarray(x0, dtype=LD)
    v0 = np.asarray(v0, dtype=LD)
    mu = LD(mu)
    dt = LD(dt)
    r0 = np.sqrt(np.dot(x0, x0))
    v2 = np.dot(v0, v0)
    a = 1 / (2 / r0 - v2 / mu)
    u = np.dot(x0, v0)
    if a > 0:
        n = np.sqrt(mu / a ** 3)
        ecosE = 1 - r0 / a
        esinE = u / np.sqrt(mu * a)
        e = np.sqrt(ecosE ** 2 + esinE ** 2)
        E0 = np.arctan2(esinE, ecosE)
        M1 = E0 - esinE + n * dt
        E1 = _bisect(lambda E: E - e * np.sin(E) - M1, M1 - e - 1, M1 + e + 1)
        dE = E1 - E0
        r1 = a * (1 - e * np.cos(E1))
        f = 1 - (a / r0) * (1 - np.cos(dE))
        g = dt - (dE - np.sin(dE)) / n
        fd = -np.sqrt(mu * a) * np.sin(dE) / (r1 * r0)
        gd = 1 - (a / r1) * (1 - np.cos(dE))
    else:
        aa = -a
        n = np.sqrt(mu / aa ** 3)
        ecoshF = 1 + r0 / aa
        esinhF = u / np.sqrt(mu * aa)
        e = np.sqrt(ecoshF ** 2 - esinhF ** 2)
        F0 = np.arcsinh(esinhF / e)
        M1 = esinhF - F0 + n * dt
        F1 = _bisect(lambda F: e * np.sinh(F) - F - M1, LD(-60), LD(60), iters=400)
        dF = F1 - F0
        r1 = aa * (e * np.cosh(F1) - 1)
        f = 1 - (aa / r0) * (np.cosh(dF) - 1)
        g = dt - (np.sinh(dF) - dF) / n
        fd = -np.sqrt(mu * aa) * np.sinh(dF) / (r1 * r0)
        gd = 1 - (aa / r1) * (np.cosh(dF) - 1)
    x1 = f * x0 + g * v0
    v1 = fd * x0 + gd * v0
    return x1.astype(np.float64), v1.astype(np.float64)


def invariants(x, v, mu):
    """Specific energy, angular momentum vector and Laplace-Runge-Lenz vector."""
    x = np.asarray(x, dtype=LD)
    v = np.asarray(v, dtype=LD)
    r = np.sqrt(np.dot(x, x))
    E = np.dot(v, v) / 2 - LD(mu) / r
    h = np.cross(x, v)
    A = np.cross(v, h) - LD(mu) * x / r
    return E, h, A
