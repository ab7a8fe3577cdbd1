"""Batched ensemble of compact planetary systems (seeded).

Recipe (the multi-simulation mode the paper mentions in Sec. 10 and Appendix B, with the GR
and tidal forces of Sec. 3 and Sec. 4 switched on):
  * star mass m_star ~ U[0.1, 1] Msun; N ~ U{8, ..., 64} planets of
    m ~ U[0.5, 10] Earth masses;
  * semi-major axes drawn log-uniform on [0.01, 0.2] AU, sorted, then pushed
    outward so that neighbours are at least 8 mutual Hill radii apart:
    a_{k+1} >= a_k (1 + 4h) / (1 - 4h), h = ((m_k + m_{k+1}) / (3 m_star))^(1/3)
    (the requested spacing does not fit inside 0.2 AU for most draws, so the
    outer edge is allowed to grow);
  * e ~ Rayleigh(0.02), i ~ Rayleigh(0.01 rad), angles uniform;
  * dt = P_inner / 20 per system;
  * tides: planets k2 = 0.3, tau = 600 s, R from 5.5 g/cm^3, rg2 = 0.33, spin
    1 rad/day along z; star k2 = 0.03, tau = 60 s, R = m_star^0.8 Rsun,
    rg2 = 0.07, spin 2 pi / 10 d along z; c = 173.1446... AU/day.
These parameter values are not given by the paper; they are stated here.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .disk import AU_CM, DAY_S, G_GAUSS, M_EARTH, SEED_BASE, elements_to_cartesian, radius_from_density

C_LIGHT = 173.1446326846693          # AU / day
R_SUN_AU = 6.957e10 / AU_CM


@dataclass
class Ensemble:
    offsets: np.ndarray     # (S+1,) int64
    x: np.ndarray           # (Ntot, 3) heliocentric
    v: np.ndarray           # (Ntot, 3) barycentric (per system)
    m: np.ndarray
    R: np.ndarray
    k2: np.ndarray
    tau: np.ndarray
    rg2: np.ndarray
    spin: np.ndarray        # (Ntot, 3) rad/day
    m_star: np.ndarray      # (S,)
    dt: np.ndarray          # (S,)
    star: np.ndarray        # (S, 8): R, k2, tau, rg2, spin x, y, z, 0
    c_light: float = C_LIGHT
    G: float = G_GAUSS

    @property
    def n_systems(self) -> int:
        return int(self.m_star.shape[0])

    def system(self, s: int) -> dict:
        a, b = int(self.offsets[s]), int(self.offsets[s + 1])
        return {"x": self.x[a:b], "v": self.v[a:b], "m": self.m[a:b], "R": self.R[a:b],
                "k2": self.k2[a:b], "tau": self.tau[a:b], "rg2": self.rg2[a:b],
                "spin": self.spin[a:b], "m_star": float(self.m_star[s]), "dt": float(self.dt[s]),
                "star": self.star[s]}


def ensemble(n_systems: int = 4096, seed: int = SEED_BASE + 3, nmin: int = 8, nmax: int = 64) -> Ensemble:
    rng = np.random.default_rng(seed)
    xs, vs, ms, Rs, ks, ts, gs, ws = [], [], [], [], [], [], [], []
    m_star = rng.uniform(0.1, 1.0, n_systems)
    dts = np.empty(n_systems)
    star = np.zeros((n_systems, 8))
    offsets = [0]
    for s in range(n_systems):
        n = int(rng.integers(nmin, nmax + 1))
        m = rng.uniform(0.5, 10.0, n) * M_EARTH
        a = np.sort(np.exp(rng.uniform(np.log(0.01), np.log(0.2), n)))
        for k in range(n - 1):
            h = ((m[k] + m[k + 1]) / (3.0 * m_star[s])) ** (1.0 / 3.0)
            a[k + 1] = max(a[k + 1], a[k] * (1 + 4 * h) / (1 - 4 * h))
        e = np.minimum(rng.rayleigh(0.02, n), 0.5)
        inc = rng.rayleigh(0.01, n)
        Om, om, M = (rng.uniform(0, 2 * np.pi, n) for _ in range(3))
        mu = G_GAUSS * (m_star[s] + m)
        x, vh = elements_to_cartesian(a, e, inc, Om, om, M, mu)
        vb = vh - (m[:, None] * vh).sum(axis=0) / (m_star[s] + m.sum())
        xs.append(x); vs.append(vb); ms.append(m)
        Rs.append(radius_from_density(m, 5.5))
        ks.append(np.full(n, 0.3)); ts.append(np.full(n, 600.0 / DAY_S)); gs.append(np.full(n, 0.33))
        w = np.zeros((n, 3)); w[:, 2] = 1.0
        ws.append(w)
        P_in = 2 * np.pi * np.sqrt(a[0] ** 3 / mu[0])
        dts[s] = P_in / 20.0
        star[s] = [m_star[s] ** 0.8 * R_SUN_AU, 0.03, 60.0 / DAY_S, 0.07, 0.0, 0.0, 2 * np.pi / 10.0, 0.0]
        offsets.append(offsets[-1] + n)
    cat = lambda L: np.ascontiguousarray(np.concatenate(L))
    return Ensemble(offsets=np.array(offsets, dtype=np.int64), x=cat(xs), v=cat(vs), m=cat(ms),
                    R=cat(Rs), k2=cat(ks), tau=cat(ts), rg2=cat(gs), spin=cat(ws), m_star=m_star,
                    dt=dts, star=star)
