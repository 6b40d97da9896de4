"""Pins of the oracle's kick-drift-kick leapfrog and energy bookkeeping.

Closed forms (two-body Kepler orbits, circular and e = 0.5) fix the
integrator's accuracy and its second-order convergence; exact properties of
KDK for central pair forces (angular momentum, time reversibility, bounded
energy error) catch a dropped half-kick, a wrong step factor or a stale
acceleration.
"""
import math

import numpy as np

from paper_2605_02744_gb300 import ics


def _circular():
    pos = np.array([[-0.5, 0.0, 0.0], [0.5, 0.0, 0.0]])
    vel = np.array([[0.0, -0.5, 0.0], [0.0, 0.5, 0.0]])
    return pos, vel, np.array([0.5, 0.5])


def _kepler_relative(t, e=0.5, a=1.0):
    """Relative position on a Kepler ellipse (GM = 1) started at pericentre."""
    M = t * math.sqrt(1.0 / a ** 3)
    E = M
    for _ in range(60):  # Newton on E - e sin E = M
        E -= (E - e * math.sin(E) - M) / (1.0 - e * math.cos(E))
    return np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])


def _eccentric():
    rp, vp = 0.5, math.sqrt(3.0)  # e = 0.5, a = 1: vp^2 = (1+e)/(a(1-e))
    pos = np.array([[-rp / 2, 0.0, 0.0], [rp / 2, 0.0, 0.0]])
    vel = np.array([[0.0, -vp / 2, 0.0], [0.0, vp / 2, 0.0]])
    return pos, vel, np.array([0.5, 0.5])


def test_circular_orbit_one_period_second_order(oracle_mod):
    pos, vel, m = _circular()
    errs = []
    for n in (200, 400):
        x, v, _, _ = oracle_mod.kdk(pos, vel, m, 0.0, 2 * math.pi / n, n)
        errs.append(np.abs(x - pos).max())
    assert errs[0] < 2e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_eccentric_orbit_matches_kepler_equation(oracle_mod):
    pos, vel, m = _eccentric()
    t = 3.0
    errs = []
    for n in (1500, 3000):
        x, _, _, _ = oracle_mod.kdk(pos, vel, m, 0.0, t / n, n)
        errs.append(np.abs((x[1] - x[0]) - _kepler_relative(t)).max())
    assert errs[0] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_energy_error_bounded_without_drift(oracle_mod):
    pos, vel, m = _eccentric()
    h = 2 * math.pi / 400
    x, v, a = pos, vel, None
    de = []
    for _ in range(10 * 400 // 50):
        x, v, a, p = oracle_mod.kdk(x, v, m, 0.0, h, 50, acc=a)
        de.append(oracle_mod.energy(v, m, p)[2])
    # exact energy for m1 = m2 = 1/2 on a relative orbit with a = 1:
    # E = -G m1 m2 / (2 a) = -1/8
    de = np.abs(np.array(de) + 0.125)
    assert de.max() < 1e-3
    first, last = de[: len(de) // 2].max(), de[len(de) // 2:].max()
    assert last < 1.5 * first


def test_angular_momentum_conserved_to_rounding(oracle_mod):
    s = ics.plummer(64, seed=3)
    x, v, _, _ = oracle_mod.kdk(s.pos, s.vel, s.mass, 0.01, 1e-3, 300)
    L0 = (s.mass[:, None] * np.cross(s.pos, s.vel)).sum(axis=0)
    L1 = (s.mass[:, None] * np.cross(x, v)).sum(axis=0)
    scale = (s.mass * np.linalg.norm(s.pos, axis=1) * np.linalg.norm(s.vel, axis=1)).sum()
    assert np.abs(L1 - L0).max() <= 1e-13 * scale
    # linear momentum too (pairwise antisymmetry)
    P1 = (s.mass[:, None] * v).sum(axis=0)
    assert np.abs(P1).max() <= 1e-14 * (s.mass * np.linalg.norm(s.vel, axis=1)).sum()


def test_time_reversibility(oracle_mod):
    s = ics.plummer(32, seed=4)
    x, v, _, _ = oracle_mod.kdk(s.pos, s.vel, s.mass, 0.01, 1e-3, 200)
    xb, vb, _, _ = oracle_mod.kdk(x, -v, s.mass, 0.01, 1e-3, 200)
    assert np.abs(xb - s.pos).max() <= 1e-12
    assert np.abs(-vb - s.vel).max() <= 1e-12


def test_fsal_restart_is_bitwise(oracle_mod):
    s = ics.plummer(100, seed=6)
    x2, v2, a2, p2 = oracle_mod.kdk(s.pos, s.vel, s.mass, 0.01, 1e-3, 7)
    x, v, a, _ = oracle_mod.kdk(s.pos, s.vel, s.mass, 0.01, 1e-3, 3)
    x, v, a, p = oracle_mod.kdk(x, v, s.mass, 0.01, 1e-3, 4, acc=a)
    assert np.array_equal(x, x2) and np.array_equal(v, v2)
    assert np.array_equal(a, a2) and np.array_equal(p, p2)


def test_energy_drift_second_order_at_plummer_1024(oracle_mod):
    # Config-1 system with 10x fewer steps: halving h cuts max |dE/E| by ~4.
    s = ics.plummer(1024, seed=0)
    _, p0 = oracle_mod.forces(s.pos, s.mass, 0.01)
    E0 = oracle_mod.energy(s.vel, s.mass, p0)[2]
    drifts = []
    for h, n in ((2e-3, 5), (1e-3, 10)):
        x, v, a = s.pos, s.vel, None
        worst = 0.0
        for _ in range(n):
            x, v, a, p = oracle_mod.kdk(x, v, s.mass, 0.01, h, 1, acc=a)
            worst = max(worst, abs(oracle_mod.energy(v, s.mass, p)[2] - E0) / abs(E0))
        drifts.append(worst)
    assert drifts[0] < 1e-5
    assert 3.0 < drifts[0] / drifts[1] < 5.0


def test_energy_sums(oracle_mod):
    vel = np.array([[1.0, 2.0, 2.0], [0.0, 0.0, 1.0]])  # |v|^2 = 9, 1
    mass = np.array([2.0, 4.0])
    pot = np.array([-1.0, -0.5])
    K, W, E = oracle_mod.energy(vel, mass, pot)
    assert (K, W, E) == (0.5 * (18 + 4), 0.5 * (-2 - 2), 11.0 - 2.0)
