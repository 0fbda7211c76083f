"""Seeded synthetic inputs: Plummer spheres, Salpeter masses, cluster batches.

This module is shared by the oracle tests and the CUDA path and holds none of
the integration method's arithmetic: it only draws initial conditions.

Workload recipe (Sect. 5 of Capuzzo-Dolcetta, Spera & Punzo, "A fully
parallel, high precision, N-body code running on hybrid computing platforms"):
particles follow the Plummer density rho(r) = 3M/(4 pi b^3) (1 + r^2/b^2)^(-5/2)
with G = M = b = 1 (Sect. 5, Plummer density and crossing-time equations).
Velocities come from the isotropic Plummer distribution function.  The systems
are then rescaled to Henon units (G = M = 1, E = -1/4).

Random numbers: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014; Vigna's public-domain reference), used
counter-based so that draw k of particle i does not depend on how many draws
other particles made:  u(seed, i, k) = top53(mix(base(seed) + (i * 2^16 + k + 1)
* GAMMA)) * 2^-53, with base(seed) = mix(seed * GAMMA).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_U64 = 0xFFFFFFFFFFFFFFFF

# Draw slots within one particle's stream.
K_RADIUS, K_COS_R, K_PHI_R, K_COS_V, K_PHI_V, K_MASS = 0, 1, 2, 3, 4, 5
K_REJECT0 = 8            # rejection pairs start here: (8, 9), (10, 11), ...
MAX_DRAWS = 1 << 16

# Plummer radius truncation: mass fraction X in (0, X_MAX].
X_MAX = 0.999
HENON_LENGTH = 3.0 * math.pi / 16.0


def mix64(z: np.ndarray) -> np.ndarray:
    """The splitmix64 output function on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_sequence(seed: int, count: int) -> np.ndarray:
    """The classic sequential splitmix64 stream: state += GAMMA; out = mix(state)."""
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & _U64) + k * GAMMA
    return mix64(state)


def _base(seed: int) -> np.uint64:
    with np.errstate(over="ignore"):
        return mix64(np.array([seed & _U64], dtype=np.uint64) * GAMMA)[0]


def uniform(seed: int, i: np.ndarray, k) -> np.ndarray:
    """Uniform doubles in [0, 1): draw k of particle stream i."""
    i = np.asarray(i, dtype=np.uint64)
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = (i << np.uint64(16)) + k + np.uint64(1)
        z = mix64(_base(seed) + ctr * GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def salpeter_masses(n: int, seed: int, m_lo: float = 0.1, m_hi: float = 100.0,
                    slope: float = 2.35) -> np.ndarray:
    """Salpeter IMF dN/dm ~ m^-slope on [m_lo, m_hi] by inverse CDF, normalised to sum 1."""
    u = uniform(seed, np.arange(n), K_MASS)
    p = 1.0 - slope
    lo, hi = m_lo ** p, m_hi ** p
    m = (lo + u * (hi - lo)) ** (1.0 / p)
    return m / m.sum()


def _isotropic(seed: int, idx: np.ndarray, k_cos: int, k_phi: int) -> np.ndarray:
    cth = 2.0 * uniform(seed, idx, k_cos) - 1.0
    phi = 2.0 * math.pi * uniform(seed, idx, k_phi)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


@dataclass
class ParticleSet:
    mass: np.ndarray   # [n]
    pos: np.ndarray    # [n, 3]
    vel: np.ndarray    # [n, 3]

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])


def plummer(n: int, seed: int, imf: str = "equal", henon: bool = True) -> ParticleSet:
    """Plummer sphere of n particles (Aarseth, Henon & Wielen 1974 sampling).

    Radius from the cumulative mass fraction X (truncated at X_MAX):
        r = (X^(-2/3) - 1)^(-1/2)  (b = 1).
    Speed q * v_esc with v_esc = sqrt(2) (1 + r^2)^(-1/4) and q drawn by von
    Neumann rejection from g(q) ~ q^2 (1 - q^2)^(7/2) (maximum below 0.1).
    Directions isotropic.  Positions and velocities are shifted to the centre
    of mass frame; with henon=True lengths are multiplied by 3 pi / 16 and
    velocities divided by sqrt(3 pi / 16) (total energy -1/4 for equal masses).
    imf: "equal" (m = 1/n) or "salpeter" (0.1-100, slope 2.35, normalised).
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    idx = np.arange(n, dtype=np.uint64)
    x_frac = X_MAX * (1.0 - uniform(seed, idx, K_RADIUS))          # (0, X_MAX]
    r = 1.0 / np.sqrt(x_frac ** (-2.0 / 3.0) - 1.0)
    pos = r[:, None] * _isotropic(seed, idx, K_COS_R, K_PHI_R)

    q = np.zeros(n)
    pending = np.arange(n)
    k = K_REJECT0
    while pending.size:
        if k + 1 >= MAX_DRAWS:
            raise RuntimeError("rejection sampling did not converge")
        qq = uniform(seed, pending, k)
        yy = 0.1 * uniform(seed, pending, k + 1)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[pending[ok]] = qq[ok]
        pending = pending[~ok]
        k += 2
    vesc = math.sqrt(2.0) * (1.0 + r * r) ** -0.25
    vel = (q * vesc)[:, None] * _isotropic(seed, idx, K_COS_V, K_PHI_V)

    if imf == "equal":
        mass = np.full(n, 1.0 / n)
    elif imf == "salpeter":
        mass = salpeter_masses(n, seed)
    else:
        raise ValueError(f"unknown imf {imf!r}")

    pos -= (mass[:, None] * pos).sum(axis=0) / mass.sum()
    vel -= (mass[:, None] * vel).sum(axis=0) / mass.sum()
    if henon:
        pos *= HENON_LENGTH
        vel /= math.sqrt(HENON_LENGTH)
    return ParticleSet(mass=mass, pos=np.ascontiguousarray(pos), vel=np.ascontiguousarray(vel))


def plummer_black_hole(n: int, seed: int, m_bh: float = 0.01, imf: str = "equal") -> ParticleSet:
    """A Plummer sphere of n - 1 stars (total mass 1, Henon units) with a massive
    central object of mass m_bh, at rest at the origin before the whole set is
    moved to its centre-of-mass frame.  The black hole is the last particle.
    The stars are not re-equilibrated: a workload with a deep central potential
    (the massive-object case of Sect. 5.5), not an equilibrium model."""
    if n < 2 or not m_bh > 0.0:
        raise ValueError("need n >= 2 and m_bh > 0")
    stars = plummer(n - 1, seed, imf)
    mass = np.concatenate([stars.mass, [m_bh]])
    pos = np.concatenate([stars.pos, np.zeros((1, 3))])
    vel = np.concatenate([stars.vel, np.zeros((1, 3))])
    mt = mass.sum()
    pos -= (mass[:, None] * pos).sum(0) / mt
    vel -= (mass[:, None] * vel).sum(0) / mt
    return ParticleSet(mass=mass, pos=np.ascontiguousarray(pos), vel=np.ascontiguousarray(vel))


def cluster_sizes(n_clusters: int, seed: int, n_lo: int = 256, n_hi: int = 16384) -> np.ndarray:
    """Cluster sizes log-uniform in [n_lo, n_hi]: round(exp(U[ln n_lo, ln n_hi]))."""
    u = uniform(seed, np.arange(n_clusters), 0)
    return np.rint(np.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))).astype(np.int64)


def cluster_batch(n_clusters: int = 512, seed: int = 4, n_lo: int = 256, n_hi: int = 16384):
    """Independent equal-mass Henon-unit Plummer clusters (cluster c uses seed 1000 + c).

    Returns (offsets[n_clusters + 1], ParticleSet of the concatenation).
    """
    sizes = cluster_sizes(n_clusters, seed, n_lo, n_hi)
    offsets = np.zeros(n_clusters + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    parts = [plummer(int(s), 1000 + c) for c, s in enumerate(sizes)]
    return offsets, ParticleSet(
        mass=np.concatenate([p.mass for p in parts]),
        pos=np.concatenate([p.pos for p in parts]),
        vel=np.concatenate([p.vel for p in parts]),
    )


def kepler_pair(e: float = 0.5, a: float = 1.0, m1: float = 0.5, m2: float = 0.5) -> ParticleSet:
    """Two bodies at pericentre of a Kepler orbit (G = 1), centre of mass at rest at the origin."""
    mt = m1 + m2
    rp = a * (1.0 - e)
    vp = math.sqrt(mt / a * (1.0 + e) / (1.0 - e))
    rel_x = np.array([rp, 0.0, 0.0])
    rel_v = np.array([0.0, vp, 0.0])
    pos = np.stack([-m2 / mt * rel_x, m1 / mt * rel_x])
    vel = np.stack([-m2 / mt * rel_v, m1 / mt * rel_v])
    return ParticleSet(mass=np.array([m1, m2]), pos=pos, vel=vel)
