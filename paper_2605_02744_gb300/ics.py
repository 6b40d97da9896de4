"""Seeded synthetic initial conditions shared by the CUDA path and the oracle.

This module holds no arithmetic of the force evaluation or of the integrator:
it only draws particle sets.  Both sides of every parity check take their
inputs from here, so it must stay free of anything the method computes.

The paper (Sec. 4.2) fixes only the particle count (409600) and the number of
steps; it gives no initial-condition distribution.  The generators below are
the synthetic stand-ins used throughout:

* ``plummer``: an equal-mass Plummer sphere in units G = M = a = 1, drawn with
  the Aarseth-Henon-Wielen (1974) recipe.  Radii come from inverting the
  cumulative mass M(<r) = r^3 (1 + r^2)^(-3/2) with X ~ U(0, 0.999) (the cut at
  0.999 keeps r <= ~38.7), directions are isotropic, the speed is q * v_esc with
  v_esc = sqrt(2) (1 + r^2)^(-1/4) and q drawn by rejection from
  g(q) = q^2 (1 - q^2)^(7/2).  The mass-weighted centre of mass is moved to the
  origin in position and velocity.
* ``plummer_lognormal``: the same phase-space sample with masses
  m_i = exp(sigma Z_i), Z ~ N(0, 1), renormalised to total mass 1 (velocities
  are not re-equilibrated for the mass spectrum).
* ``batched_plummer``: 512 independent clusters with N_c log-uniform in
  [64, 8192], each a unit-mass Plummer sphere, concatenated with CSR offsets.
* ``perturb_positions``: Gaussian displacement used to make an adjoint target.

Random draws use numpy's PCG64 (``default_rng``) in the fixed order documented
in each function; the arrays are generated once and handed to both paths.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "ParticleSet",
    "plummer",
    "plummer_lognormal",
    "batched_sizes",
    "batched_plummer",
    "perturb_positions",
    "random_coordinates",
]

# Largest X drawn for the cumulative-mass inversion (radius cut ~38.7 a).
_X_MAX = 0.999


@dataclass
class ParticleSet:
    """FP64 particle arrays: pos [N,3], vel [N,3], mass [N] (C-contiguous)."""

    pos: np.ndarray
    vel: np.ndarray
    mass: np.ndarray
    offsets: np.ndarray | None = None  # CSR offsets [B+1] for batched sets

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """Unit vectors uniform on the sphere: cos(theta) ~ U(-1,1), phi ~ U(0,2pi)."""
    cth = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def _plummer_q(rng: np.random.Generator, n: int) -> np.ndarray:
    """Speed fractions q in [0,1) by rejection from g(q) = q^2 (1-q^2)^(7/2).

    The maximum of g is ~0.0920 (at q^2 = 2/9), so the envelope U(0, 0.1)
    bounds it.  Candidates are drawn in blocks of 2n pairs (q, y), q first.
    """
    out = np.empty(n)
    filled = 0
    while filled < n:
        m = 2 * (n - filled) + 16
        q = rng.uniform(0.0, 1.0, m)
        y = rng.uniform(0.0, 0.1, m)
        ok = q[y < q * q * (1.0 - q * q) ** 3.5]
        take = min(ok.size, n - filled)
        out[filled:filled + take] = ok[:take]
        filled += take
    return out


def _plummer_phase_space(rng: np.random.Generator, n: int):
    """Radius, then position direction, then q, then velocity direction."""
    x = rng.uniform(0.0, _X_MAX, n)
    r = 1.0 / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
    pos = r[:, None] * _isotropic(rng, n)
    q = _plummer_q(rng, n)
    vesc = math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    vel = (q * vesc)[:, None] * _isotropic(rng, n)
    return pos, vel


def _to_com_frame(pos, vel, mass):
    mtot = mass.sum()
    pos = pos - (mass[:, None] * pos).sum(axis=0) / mtot
    vel = vel - (mass[:, None] * vel).sum(axis=0) / mtot
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel)


def plummer(n: int, seed: int = 0) -> ParticleSet:
    """Equal-mass Plummer sphere, G = M = a = 1, masses 1/n."""
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.default_rng(seed)
    pos, vel = _plummer_phase_space(rng, n)
    mass = np.full(n, 1.0 / n)
    pos, vel = _to_com_frame(pos, vel, mass)
    return ParticleSet(pos, vel, mass)


def plummer_lognormal(n: int, seed: int = 0, sigma: float = 0.5) -> ParticleSet:
    """Plummer phase space (same draws as ``plummer``) with log-normal masses.

    Z is drawn from a second generator seeded with [seed, 1] so the phase-space
    sample equals the equal-mass one for the same seed.
    """
    rng = np.random.default_rng(seed)
    pos, vel = _plummer_phase_space(rng, n)
    z = np.random.default_rng([seed, 1]).standard_normal(n)
    mass = np.exp(sigma * z)
    mass /= mass.sum()
    pos, vel = _to_com_frame(pos, vel, mass)
    return ParticleSet(pos, vel, np.ascontiguousarray(mass))


def batched_sizes(b: int = 512, seed: int = 1, nmin: int = 64, nmax: int = 8192) -> np.ndarray:
    """Cluster sizes log-uniform in [nmin, nmax]: round(exp(U(ln nmin, ln nmax)))."""
    u = np.random.default_rng(seed).uniform(math.log(nmin), math.log(nmax), b)
    return np.clip(np.rint(np.exp(u)), nmin, nmax).astype(np.int64)


def batched_plummer(b: int = 512, seed: int = 1, nmin: int = 64, nmax: int = 8192,
                    sizes: np.ndarray | None = None) -> ParticleSet:
    """Independent unit-mass Plummer clusters, concatenated, with CSR offsets.

    Cluster c is drawn from ``SeedSequence(seed).spawn(b)[c]``; each has its
    own centre of mass at the origin (clusters do not interact).
    """
    if sizes is None:
        sizes = batched_sizes(b, seed, nmin, nmax)
    sizes = np.asarray(sizes, dtype=np.int64)
    b = int(sizes.shape[0])
    children = np.random.SeedSequence(seed).spawn(b)
    pos, vel, mass = [], [], []
    for c in range(b):
        rng = np.random.default_rng(children[c])
        n = int(sizes[c])
        p, v = _plummer_phase_space(rng, n)
        m = np.full(n, 1.0 / n)
        p, v = _to_com_frame(p, v, m)
        pos.append(p)
        vel.append(v)
        mass.append(m)
    offsets = np.zeros(b + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    return ParticleSet(np.ascontiguousarray(np.concatenate(pos)),
                       np.ascontiguousarray(np.concatenate(vel)),
                       np.ascontiguousarray(np.concatenate(mass)), offsets)


def perturb_positions(pos: np.ndarray, std: float = 1e-3, seed: int = 2) -> np.ndarray:
    """pos + N(0, std^2) per coordinate (std is a standard deviation)."""
    d = np.random.default_rng(seed).normal(0.0, std, pos.shape)
    return np.ascontiguousarray(pos + d)


def random_coordinates(n: int, k: int = 64, seed: int = 3) -> np.ndarray:
    """k distinct flat indices into the 7n scalars (3n pos, 3n vel, n mass)."""
    return np.sort(np.random.default_rng(seed).choice(7 * n, size=k, replace=False))
