"""Planetesimal-disk and ring workloads (numpy, seeded).

Units: AU, day, solar mass.  G = k^2 with the Gaussian constant k.

Disk recipe (the planetesimal disks of the paper's performance and
higher-level-changeover tests, Sec. 6.3-6.5 and Sec. 9: N equal-mass bodies between
a_min and a_max with surface density proportional to a^-1.5):
  * a drawn so that dN/da ~ a^-0.5:  a = (sqrt(a_min) + u (sqrt(a_max) - sqrt(a_min)))^2
  * e ~ Rayleigh(sigma_e), i ~ Rayleigh(sigma_i) [rad], Omega, omega, M ~ U[0, 2pi)
  * equal masses m = M_disk / N, optional embryos at a ~ U[a_min, a_max]
  * elements -> heliocentric Cartesian with mu_i = G (m_star + m_i)
  * velocities made barycentric: v_i = v_hel,i - sum_j m_j v_hel,j / (m_star + sum_j m_j)
  * physical radius from the bulk density (2 g/cm^3 by default)

Ring recipe (the close-encounter performance test, Sec. 6.2): N equal masses
regularly spaced on a circle, on circular orbits; the critical radius is chosen
so that every body has eight encounter partners (all others for N < 16).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

K_GAUSS = 0.01720209895
G_GAUSS = K_GAUSS * K_GAUSS          # AU^3 / (Msun day^2)
M_EARTH = 1.0 / 332946.0487           # Msun
MSUN_G = 1.98847e33                   # g
AU_CM = 1.495978707e13                # cm
DAY_S = 86400.0

SEED_BASE = 20110058


@dataclass
class Workload:
    """Initial state and integrator parameters of one synthetic run."""
    name: str
    x: np.ndarray          # (N,3) heliocentric positions [AU]
    v: np.ndarray          # (N,3) barycentric velocities [AU/day]
    m: np.ndarray          # (N,) masses [Msun]
    R: np.ndarray          # (N,) physical radii [AU]
    m_star: float = 1.0
    G: float = G_GAUSS
    dt: float = 6.0875
    n1: float = 3.0
    n2: float = 0.4
    f_pc: float = 4.0
    slevels: int = 1
    substeps: int = 1
    nsteps: int = 100
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.m.shape[0])


def _kepler_E(M: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Eccentric anomaly from the mean anomaly (Newton, vectorised, e < 1)."""
    E = M + e * np.sin(M)
    for _ in range(50):
        f = E - e * np.sin(E) - M
        fp = 1.0 - e * np.cos(E)
        dE = f / fp
        E = E - dE
        if np.max(np.abs(dE)) < 1e-15:
            break
    return E


def elements_to_cartesian(a, e, inc, Om, om, M, mu):
    """Heliocentric position/velocity from Keplerian elements (elliptic)."""
    E = _kepler_E(M, e)
    cE, sE = np.cos(E), np.sin(E)
    b = a * np.sqrt(1.0 - e * e)
    # perifocal frame
    xp = a * (cE - e)
    yp = b * sE
    n = np.sqrt(mu / a ** 3)
    Edot = n / (1.0 - e * cE)
    vxp = -a * sE * Edot
    vyp = b * cE * Edot
    cO, sO = np.cos(Om), np.sin(Om)
    co, so = np.cos(om), np.sin(om)
    ci, si = np.cos(inc), np.sin(inc)
    P = np.stack([cO * co - sO * so * ci, sO * co + cO * so * ci, so * si], axis=-1)
    Q = np.stack([-cO * so - sO * co * ci, -sO * so + cO * co * ci, co * si], axis=-1)
    x = xp[:, None] * P + yp[:, None] * Q
    v = vxp[:, None] * P + vyp[:, None] * Q
    return x, v


def radius_from_density(m, rho_cgs):
    """Physical radius [AU] of a sphere of mass m [Msun] and density rho [g/cm^3]."""
    vol = (m * MSUN_G) / rho_cgs
    return (3.0 * vol / (4.0 * np.pi)) ** (1.0 / 3.0) / AU_CM


def disk(n: int, a_min: float, a_max: float, m_disk_earth: float, seed: int,
         n_embryos: int = 0, m_embryo_earth: float = 0.1, sigma_e: float = 0.01,
         sigma_i: float = 0.005, rho: float = 2.0, m_star: float = 1.0,
         name: str = "disk", **params) -> Workload:
    """Equal-mass planetesimal disk (plus optional embryos), see module doc."""
    rng = np.random.default_rng(seed)
    ntot = n + n_embryos
    u = rng.random(n)
    sa, sb = np.sqrt(a_min), np.sqrt(a_max)
    a = (sa + u * (sb - sa)) ** 2
    m = np.full(n, m_disk_earth * M_EARTH / n)
    if n_embryos:
        a = np.concatenate([a, rng.uniform(a_min, a_max, n_embryos)])
        m = np.concatenate([m, np.full(n_embryos, m_embryo_earth * M_EARTH)])
    e = rng.rayleigh(sigma_e, ntot)
    e = np.minimum(e, 0.9)
    inc = rng.rayleigh(sigma_i, ntot)
    Om = rng.uniform(0.0, 2 * np.pi, ntot)
    om = rng.uniform(0.0, 2 * np.pi, ntot)
    M = rng.uniform(0.0, 2 * np.pi, ntot)
    mu = G_GAUSS * (m_star + m)
    x, vh = elements_to_cartesian(a, e, inc, Om, om, M, mu)
    vb = vh - (m[:, None] * vh).sum(axis=0) / (m_star + m.sum())
    R = radius_from_density(m, rho)
    return Workload(name=name, x=np.ascontiguousarray(x), v=np.ascontiguousarray(vb),
                    m=m, R=R, m_star=m_star, **params)


def ring(n: int, r: float = 1.0, m_body_earth: float = 0.01, dt: float = 6.0875,
         partners: int = 8, m_star: float = 1.0) -> Workload:
    """Ring of n equal masses on circular orbits at radius r (Sec. 6.2 test).

    The critical radius comes from the velocity term only (n1 = 0) with n2 set
    so that rc lies between the (partners/2)-th and the next neighbour's chord:
    each body then has `partners` neighbours within rc (all others when
    n < 2 partners, i.e. N < 16 for the paper's eight).
    """
    phi = 2 * np.pi * np.arange(n) / n
    x = np.stack([r * np.cos(phi), r * np.sin(phi), np.zeros(n)], axis=-1)
    m = np.full(n, m_body_earth * M_EARTH)
    vc = np.sqrt(G_GAUSS * (m_star + m) / r)
    vh = np.stack([-vc * np.sin(phi), vc * np.cos(phi), np.zeros(n)], axis=-1)
    vb = vh - (m[:, None] * vh).sum(axis=0) / (m_star + m.sum())
    spacing = 2 * r * np.sin(np.pi / n)
    half = partners // 2
    if n < 2 * partners:
        rc = 2.0 * r * 1.01          # everyone sees everyone (N < 16 for eight partners)
    else:
        # between the half-th and (half+1)-th neighbour chord lengths
        c_in = 2 * r * np.sin(np.pi * half / n)
        c_out = 2 * r * np.sin(np.pi * (half + 1) / n)
        rc = 0.5 * (c_in + c_out)
    speed = np.sqrt((vb * vb).sum(axis=1)).min()
    n2 = rc / (dt * speed)
    R = radius_from_density(m, 2.0)
    return Workload(name=f"ring{n}", x=x, v=vb, m=m, R=R, m_star=m_star, dt=dt, n1=0.0,
                    n2=float(n2), f_pc=1.5, extra={"rc_target": rc, "spacing": spacing})


# ---------------------------------------------------------------------------
# The five benchmark configurations (seed = SEED_BASE + index).

def config_workload(index: int, n_override: int | None = None) -> Workload:
    """Workload of configuration `index` (0..2: disks; see module doc)."""
    seed = SEED_BASE + index
    if index == 0:
        n = n_override or 2048
        return disk(n, 0.5, 2.0, 2.0, seed, name=f"disk{n}_a0.5-2_2Me", nsteps=100)
    if index == 1:
        n = n_override or 16384
        return disk(n, 0.5, 2.0, 2.0, seed, name=f"disk{n}_a0.5-2_2Me", nsteps=1000)
    if index == 2:
        n = n_override or 65536
        return disk(n, 0.5, 4.0, 5.0, seed, n_embryos=4, m_embryo_earth=0.1,
                    name=f"disk{n}+4emb_a0.5-4_5Me", slevels=2, substeps=10, nsteps=1000)
    if index == 4:
        n = n_override or 4096
        return disk(n, 0.5, 2.0, 2.0, seed, name=f"disk{n}_a0.5-2_2Me", nsteps=1000)
    raise ValueError(f"no disk workload for configuration {index}")
