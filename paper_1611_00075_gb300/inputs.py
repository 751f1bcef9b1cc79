"""Seeded synthetic inputs shaped like the paper's benchmark systems.

This module holds no arithmetic of the MD method itself: it only lays atoms on
fcc lattices, carves voids, and draws Maxwell-Boltzmann velocities.  Both the
CUDA path (through tests and ``bench.py``) and the CPU oracle consume what it
returns, so it must stay free of anything either side computes.

The paper's own configurations (Cu105, Porous, Fe126, Cu144, PnC; Sec. 3.1)
are not available, so these stand in for them:

* ``lj_fcc``      -- homogeneous bulk crystal (stands in for Cu105 / Cu144)
* ``lj_porous``   -- fcc solid with random spherical voids (stands in for the
  inhomogeneous Porous and PnC systems)
* ``sc_fcc``      -- many-body fcc metal at its lattice constant
* ``eam_bcc``     -- bcc metal under a piecewise embedded-atom potential
  (stands in for Fe126)
* ``lj_alloy``, ``lj_layer`` -- a Cu-Au-like binary LJ crystal, random or in
  slabs (stand in for the Alloy and Layer systems)
* ``lj_ensemble`` -- a batch of independent replicas of uneven size

Random numbers come from splitmix64 (Steele, Lea & Flood 2014): output k of a
stream seeded with s is mix(s + (k + 1) * 0x9E3779B97F4A7C15) with the
published mixing constants.  Gaussians use the Box-Muller transform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1611000075
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
BCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the splitmix64 stream `seed`."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in (0, 1): ((z >> 11) + 0.5) * 2^-53."""
    z = splitmix64(seed, count, offset)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def gaussian(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal deviates by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m, 2 * offset)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    t = 2.0 * math.pi * u[1::2]
    g = np.empty(2 * m)
    g[0::2] = r * np.cos(t)
    g[1::2] = r * np.sin(t)
    return g[:count]


def fcc_lattice(nc, a0: float, basis=FCC_BASIS) -> np.ndarray:
    """Sites a0 * (cell + basis_k) of an nc[0] x nc[1] x nc[2] fcc block,
    ordered by (ix, iy, iz, k)."""
    nx, ny, nz = (nc, nc, nc) if np.isscalar(nc) else nc
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ix, iy, iz], axis=-1).reshape(-1, 1, 3).astype(np.float64)
    pos = a0 * (cells + basis[None, :, :])
    return np.ascontiguousarray(pos.reshape(-1, 3))


def bcc_lattice(nc, a0: float) -> np.ndarray:
    """Sites a0 * (cell + basis_k) of a bcc block, ordered by (ix, iy, iz, k)."""
    return fcc_lattice(nc, a0, BCC_BASIS)


def maxwell_boltzmann(n: int, T: float, mass: float, seed: int) -> np.ndarray:
    """Gaussian velocities with variance T/m per component, zero total
    momentum, rescaled so that KE = (3n - 3) T / 2 exactly (the temperature
    is counted over 3n - 3 degrees of freedom)."""
    v = gaussian(seed, 3 * n).reshape(n, 3) * math.sqrt(T / mass)
    if n == 0:
        return v
    return rescale_velocities(v, T, mass)


def rescale_velocities(v, T: float, mass: float = 1.0) -> np.ndarray:
    """Velocities with the mean momentum removed and scaled so that
    KE = (3n - 3) T / 2 exactly (the temperature over 3n - 3 degrees of
    freedom); zero for T = 0 or a single atom."""
    v = np.array(v, dtype=np.float64).reshape(-1, 3)
    n = v.shape[0]
    v -= v.mean(axis=0, keepdims=True)
    if n > 1 and T > 0:
        ke = 0.5 * mass * float(np.sum(v * v))
        v *= math.sqrt(0.5 * (3 * n - 3) * T / ke)
    else:
        v[:] = 0.0
    return np.ascontiguousarray(v)


# The liquid of config 2 is melted from fcc: the crystal is heated past its
# stability limit at T* = 2.4, then held at the target T* = 1.2, velocities
# rescaled to the stage's temperature every MELT_RESCALE_EVERY steps (and once
# more at the end).  Whatever runs the steps -- the oracle for test inputs, the
# GPU path for the benchmark's own input -- follows this schedule.
MELT_SCHEDULE = ((2.4, 1000), (1.2, 1000))  # (T*, steps) per stage: 2,000 steps
MELT_RESCALE_EVERY = 50

# Equilibration of the porous solid before it is measured, in the same form:
# the crystal with carved voids relaxes its surfaces and heats (run without
# rescaling from T* 0.3 it settles near T* 0.4 within about 600 steps, its
# rebuild rate rising from 9 to 12 per 100 steps); held at T* 0.3 by the
# rescaling for 1,000 steps it reaches its steady rebuild rate.
POROUS_EQUIL_SCHEDULE = ((0.3, 1000),)


def tile(s: "System", k: int) -> "System":
    """k x k x k periodic copies of a cubic system (atoms of copy (a, b, c),
    a slowest, follow each other); velocities are copied unchanged."""
    off = np.array([(a, b, c) for a in range(k) for b in range(k) for c in range(k)],
                   dtype=np.float64) * s.box
    pos = (s.pos[None, :, :] + off[:, None, :]).reshape(-1, 3)
    vel = np.tile(s.vel, (k ** 3, 1))
    return System("%s_x%d" % (s.name, k), np.ascontiguousarray(pos), np.ascontiguousarray(vel),
                  s.box * k, dict(s.params))


def carve_voids(nc: int, a0: float, fraction: float, rmin: float, rmax: float,
                seed: int) -> np.ndarray:
    """Boolean keep-mask over the sites of fcc_lattice(nc, a0): spherical
    voids with centres uniform in the periodic box and radii uniform in
    [rmin, rmax] are added one at a time until at least `fraction` of the
    sites lie inside some void (periodic distance < radius)."""
    L = nc * a0
    nsite = 4 * nc ** 3
    keep = np.ones(nsite, dtype=bool)
    removed = 0
    target = math.ceil(fraction * nsite)
    v = 0
    while removed < target:
        u = uniform(seed, 4, 4 * v)
        v += 1
        c = u[:3] * L
        r = rmin + (rmax - rmin) * u[3]
        # candidate cells: the bounding cube of the sphere, wrapped
        rng = []
        for d in range(3):
            lo = math.floor((c[d] - r) / a0) - 1
            hi = math.floor((c[d] + r) / a0) + 1
            idx = np.arange(lo, hi + 1) % nc
            rng.append(np.unique(idx))
        ix, iy, iz = np.meshgrid(rng[0], rng[1], rng[2], indexing="ij")
        cell = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=-1)
        site = a0 * (cell[:, None, :].astype(np.float64) + FCC_BASIS[None, :, :])
        d = site - c
        d -= L * np.round(d / L)
        inside = np.sum(d * d, axis=-1) < r * r
        lin = ((cell[:, 0] * nc + cell[:, 1]) * nc + cell[:, 2])[:, None] * 4 + np.arange(4)
        hit = lin[inside]
        newly = keep[hit]
        removed += int(np.count_nonzero(newly))
        keep[hit] = False
    return keep


@dataclass
class System:
    """One synthetic system: positions/velocities are n x 3 float64 in
    original atom order; `params` holds the potential and integrator
    settings by name."""
    name: str
    pos: np.ndarray
    vel: np.ndarray
    box: np.ndarray
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def lj_fcc(nc: int = 10, rho: float = 0.8442, T: float = 0.72, seed: int = SEED_BASE + 1,
           rc: float = 2.5, skin: float = 0.3, dt: float = 0.005) -> System:
    """Lennard-Jones fcc crystal of nc^3 cells at reduced density rho."""
    a0 = (4.0 / rho) ** (1.0 / 3.0)
    pos = fcc_lattice(nc, a0)
    vel = maxwell_boltzmann(pos.shape[0], T, 1.0, seed)
    box = np.full(3, nc * a0)
    return System("lj_fcc_%d" % nc, pos, vel, box,
                  dict(potential="lj", eps=1.0, sigma=1.0, rc=rc, skin=skin, dt=dt, mass=1.0,
                       T=T, rho=rho))


def lj_porous(nc: int = 160, rho: float = 0.8442, T: float = 0.3, fraction: float = 0.40,
              rmin: float = 3.0, rmax: float = 15.0, seed: int = SEED_BASE + 3,
              rc: float = 2.5, skin: float = 0.3, dt: float = 0.005) -> System:
    """Porous LJ solid: fcc sites minus random spherical voids."""
    a0 = (4.0 / rho) ** (1.0 / 3.0)
    keep = carve_voids(nc, a0, fraction, rmin, rmax, seed)
    pos = np.ascontiguousarray(fcc_lattice(nc, a0)[keep])
    vel = maxwell_boltzmann(pos.shape[0], T, 1.0, seed + 1000)
    box = np.full(3, nc * a0)
    return System("lj_porous_%d" % nc, pos, vel, box,
                  dict(potential="lj", eps=1.0, sigma=1.0, rc=rc, skin=skin, dt=dt, mass=1.0,
                       T=T, rho=rho, sites=4 * nc ** 3))


# Sutton-Chen parameters of the many-body benchmark (eps = a = 1, c, n, m),
# the temperature equivalent of 300 K and the time step equivalent of 2 fs for
# Sutton-Chen copper (eps = 1.2382e-2 eV, a = 3.61 A, m = 63.546 u).
SC_DEFAULT = dict(eps=1.0, a=1.0, c=39.432, n_exp=9.0, m_exp=6.0, rc=2.0, skin=0.2,
                  T=2.088, dt=7.6e-4, mass=1.0)


def sc_fcc(nc: int = 128, a0: float = 1.0, seed: int = SEED_BASE + 4, **over) -> System:
    p = dict(SC_DEFAULT)
    p.update(over)
    pos = fcc_lattice(nc, a0)
    vel = maxwell_boltzmann(pos.shape[0], p["T"], p["mass"], seed)
    box = np.full(3, nc * a0)
    return System("sc_fcc_%d" % nc, pos, vel, box,
                  dict(potential="sc", eps=p["eps"], sigma=p["a"], c=p["c"], n_exp=p["n_exp"],
                       m_exp=p["m_exp"], rc=p["rc"], skin=p["skin"], dt=p["dt"],
                       mass=p["mass"], T=p["T"]))


# A synthetic many-body metal with the piecewise embedded-atom form of the
# paper's Fe potential (its tables are not public here): bcc with a0 = 1,
# pair and density functions that are sums of truncated cubics on knots
# (Phi: seven knots, psi: one), F(rho) = -F_sqrt sqrt(rho) + F_quad rho^2.
# The pair knots' coefficients were fitted to a Morse shape (depth 0.25,
# stiffness 4.5) whose minimum was placed so that the bcc lattice with
# a0 = 1 sits at its energy minimum (cohesive energy -3.008 per atom); the
# cutoff 1.8 keeps shells 1-5 (58 neighbours).  T* = 0.018 is the ratio of
# 300 K to iron's cohesive energy (0.026 / 4.28 eV) times 3.008.
EAM_FE_LIKE = dict(phi_r=(0.9, 1.05, 1.2, 1.35, 1.5, 1.65, 1.8),
                   phi_a=(160.6, -23.87, 26.45, -11.78, 5.545, -1.215, -0.5516),
                   psi_r=(1.8,), psi_a=(1.0,), F_sqrt=0.5, F_quad=0.0,
                   rc=1.8, skin=0.15, T=0.018, dt=0.002, mass=1.0)


def eam_bcc(nc: int = 126, a0: float = 1.0, seed: int = SEED_BASE + 6, **over) -> System:
    """bcc crystal of nc^3 cells (2 nc^3 atoms) under the piecewise EAM
    (126^3 cells: 4,000,752 atoms, the size of the paper's Fe126)."""
    p = dict(EAM_FE_LIKE)
    p.update(over)
    pos = bcc_lattice(nc, a0)
    vel = maxwell_boltzmann(pos.shape[0], p["T"], p["mass"], seed)
    box = np.full(3, nc * a0)
    return System("eam_bcc_%d" % nc, pos, vel, box, dict(potential="eam", **p))


# A synthetic Cu-Au-like binary Lennard-Jones system standing in for the
# paper's Alloy (Cu75Au25) and Layer (Cu and Au slabs) configurations, whose
# Cleri-Rosato parameters are not available here.  Species 0 (Cu-like):
# eps = sigma = mass = 1; species 1 (Au-like): eps 1.12, sigma 1.128, mass
# 3.10 -- the Au/Cu ratios of published Lennard-Jones fits for the two fcc
# metals and of their atomic masses; unlike pairs by Lorentz-Berthelot
# mixing.  fcc lattice constant 1.625, the minimum of the unrelaxed random
# 25 % alloy's lattice energy; T* = 0.063 (300 K over the Cu-like eps,
# 0.409 eV).  The unrelaxed unlike neighbours are compressed (Au-like pairs at
# 1.01 sigma), which stiffens the dynamics: dt = 0.002 keeps the float64
# energy within 1e-5 over 400 steps (0.005 drifts by 5e-5).
LJ_CUAU = dict(eps=(1.0, 1.12), sigma=(1.0, 1.128), mass=(1.0, 3.10), a0=1.625,
               rc=2.5, skin=0.3, dt=0.002, T=0.063)


def mixing_rules(eps, sigma):
    """nt x nt pair parameters: sqrt(eps_a eps_b) and (sigma_a + sigma_b) / 2."""
    e = np.sqrt(np.outer(eps, eps))
    s = 0.5 * (np.add.outer(sigma, sigma))
    return e, s


def _typed_system(name, pos, types, box, p, seed):
    mass = np.asarray(p["mass"])[types]
    # Maxwell-Boltzmann per species mass: unit Gaussians scaled by 1/sqrt(m),
    # then the common shift and rescale to exactly T (momentum-weighted)
    g = gaussian(seed, 3 * len(pos)).reshape(-1, 3) * np.sqrt(p["T"] / mass)[:, None]
    g -= (mass[:, None] * g).sum(axis=0) / mass.sum()
    ke = 0.5 * float(np.sum(mass[:, None] * g * g))
    g *= math.sqrt(0.5 * (3 * len(pos) - 3) * p["T"] / ke)
    t_eps, t_sigma = mixing_rules(p["eps"], p["sigma"])
    params = dict(potential="lj", rc=p["rc"], skin=p["skin"], dt=p["dt"], T=p["T"],
                  types=np.ascontiguousarray(types, np.int32), t_eps=t_eps, t_sigma=t_sigma,
                  t_mass=np.asarray(p["mass"], np.float64), eps=1.0, sigma=1.0, mass=1.0)
    return System(name, np.ascontiguousarray(pos), np.ascontiguousarray(g), box, params)


def lj_alloy(nc: int = 105, frac: float = 0.25, seed: int = SEED_BASE + 7, **over) -> System:
    """Random substitutional alloy: fcc sites of nc^3 cells, each Au-like with
    probability frac (105^3 cells: 4,630,500 atoms, the paper's Alloy size)."""
    p = dict(LJ_CUAU)
    p.update(over)
    pos = fcc_lattice(nc, p["a0"])
    types = (uniform(seed, len(pos)) < frac).astype(np.int32)
    return _typed_system("lj_alloy_%d" % nc, pos, types, np.full(3, nc * p["a0"]), p, seed + 1)


def lj_layer(nc: int = 99, slab: int = 9, seed: int = SEED_BASE + 8, **over) -> System:
    """Slabs of slab fcc cells along z, alternately Cu-like and Au-like
    (99^3 cells: 3,881,196 atoms, near the paper's Layer size)."""
    p = dict(LJ_CUAU)
    p.update(over)
    pos = fcc_lattice(nc, p["a0"])
    nz = np.repeat(np.arange(nc), 4)  # the fcc order is (ix, iy, iz, basis)
    iz = np.tile(nz, nc * nc)
    types = ((iz // slab) % 2).astype(np.int32)
    return _typed_system("lj_layer_%d" % nc, pos, types, np.full(3, nc * p["a0"]), p, seed + 1)


def lj_ensemble(count: int = 64, nmin: int = 1000, nmax: int = 200000,
                seed: int = SEED_BASE + 5, rc: float = 2.5, skin: float = 0.3,
                dt: float = 0.005, min_cells: int = 6):
    """Replicas with sizes log-uniform in [nmin, nmax]: n_c = max(min_cells,
    round((N*/4)^(1/3))) fcc cells per side, rho uniform in [0.7, 0.9],
    T uniform in [0.5, 1.5]."""
    u = uniform(seed, 3 * count).reshape(count, 3)
    out = []
    for r in range(count):
        nstar = math.exp(math.log(nmin) + (math.log(nmax) - math.log(nmin)) * u[r, 0])
        nc = max(min_cells, int(round((nstar / 4.0) ** (1.0 / 3.0))))
        rho = 0.7 + 0.2 * u[r, 1]
        T = 0.5 + 1.0 * u[r, 2]
        out.append(lj_fcc(nc=nc, rho=rho, T=T, seed=seed + 100 + r, rc=rc, skin=skin, dt=dt))
    return out
