"""Pins of the oracle's jerk (App. A, Algorithm 3) and fourth-order Hermite.

The jerk is the time derivative of the acceleration along the motion, so it
must equal the central difference (a(x + h v) - a(x - h v)) / (2h) of the
oracle's independent acceleration code; a two-body case is worked by hand;
the integrator must converge at fourth order on a Kepler ellipse (error
ratio ~16 when the step halves) and conserve energy far better than
leapfrog at the same step.
"""
import math

import numpy as np

from paper_2605_02744_gb300 import ics


def test_jerk_is_directional_derivative_of_acceleration(oracle_mod):
    for eps in (0.0, 0.02):
        s = ics.plummer_lognormal(200, seed=3)
        a, j, p = oracle_mod.forces_jerk(s.pos, s.vel, s.mass, eps)
        h = 1e-6
        ap, _ = oracle_mod.forces(s.pos + h * s.vel, s.mass, eps)
        am, _ = oracle_mod.forces(s.pos - h * s.vel, s.mass, eps)
        fd = (ap - am) / (2 * h)
        assert np.abs(j - fd).max() <= 1e-7 * np.abs(j).max()
        a0, p0 = oracle_mod.forces(s.pos, s.mass, eps)
        assert np.array_equal(a, a0) and np.array_equal(p, p0)


def test_two_body_jerk_by_hand(oracle_mod):
    # j at the origin from m=2 at (3,4,0) moving with (0,0,1): d.w = 0, so
    # jerk = 2 (0,0,1) / 125
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    vel = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    _, j, _ = oracle_mod.forces_jerk(pos, vel, np.array([1.0, 2.0]), 0.0)
    np.testing.assert_allclose(j[0], [0.0, 0.0, 2.0 / 125.0], rtol=1e-15, atol=1e-18)
    # radial motion: w = (3,4,0)/5 along d, d.w = 5: jerk = 2 (w/125 - 3*5*d/3125)
    vel = np.array([[0.0, 0.0, 0.0], [0.6, 0.8, 0.0]])
    _, j, _ = oracle_mod.forces_jerk(pos, vel, np.array([1.0, 2.0]), 0.0)
    exp = 2.0 * (np.array([0.6, 0.8, 0.0]) / 125.0 - 15.0 * np.array([3.0, 4.0, 0.0]) / 3125.0)
    np.testing.assert_allclose(j[0], exp, rtol=1e-14, atol=1e-18)


def _kepler_relative(t, e=0.5, a=1.0):
    M = t * math.sqrt(1.0 / a ** 3)
    E = M
    for _ in range(60):
        E -= (E - e * math.sin(E) - M) / (1.0 - e * math.cos(E))
    return np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])


def test_hermite4_fourth_order_on_kepler_ellipse(oracle_mod):
    rp, vp = 0.5, math.sqrt(3.0)
    pos = np.array([[-rp / 2, 0.0, 0.0], [rp / 2, 0.0, 0.0]])
    vel = np.array([[0.0, -vp / 2, 0.0], [0.0, vp / 2, 0.0]])
    m = np.array([0.5, 0.5])
    t = 3.0
    errs = []
    for n in (300, 600):
        x, _, _, _ = oracle_mod.hermite4(pos, vel, m, 0.0, t / n, n)
        errs.append(np.abs((x[1] - x[0]) - _kepler_relative(t)).max())
    assert errs[0] < 1e-5
    assert 12.0 < errs[0] / errs[1] < 20.0


def test_hermite4_energy_beats_leapfrog(oracle_mod):
    s = ics.plummer(128, seed=2)
    eps, h, n = 0.05, 1e-2, 50
    _, p0 = oracle_mod.forces(s.pos, s.mass, eps)
    E0 = oracle_mod.energy(s.vel, s.mass, p0)[2]
    xh, vh, _, _ = oracle_mod.hermite4(s.pos, s.vel, s.mass, eps, h, n)
    _, ph = oracle_mod.forces(xh, s.mass, eps)
    xl, vl, _, pl = oracle_mod.kdk(s.pos, s.vel, s.mass, eps, h, n)
    dh = abs(oracle_mod.energy(vh, s.mass, ph)[2] - E0)
    dl = abs(oracle_mod.energy(vl, s.mass, pl)[2] - E0)
    assert dh < 0.1 * dl


def test_jerk_rows_equal_full(oracle_mod):
    s = ics.plummer(700, seed=4)
    a, j, _ = oracle_mod.forces_jerk(s.pos, s.vel, s.mass, 0.01)
    rows = np.array([3, 699, 0, 3])
    ar, jr = oracle_mod.forces_jerk_rows(s.pos, s.vel, s.mass, 0.01, rows)
    assert np.array_equal(ar, a[rows]) and np.array_equal(jr, j[rows])
