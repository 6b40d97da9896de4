"""Pins of the FP64 oracle's force and potential (Eq. 1, Sec. 2.1).

Each test checks the oracle against something it cannot reproduce by
re-running its own arithmetic: 50-digit arithmetic, numbers worked out by
hand, exact invariants (Newton's third law, symmetries, exact power-of-two
scaling) and the continuum Plummer field.
"""
import math

import numpy as np
import pytest

from oracle import hiprec
from paper_2605_02744_gb300 import ics


def _rand_system(n, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    pos = rng.normal(0.0, spread, (n, 3))
    mass = rng.uniform(0.1, 2.0, n)
    return pos, mass


@pytest.mark.parametrize("n", [2, 3, 5, 8])
@pytest.mark.parametrize("eps", [0.0, 0.01, 0.7])
def test_matches_50_digit_brute_force(oracle_mod, n, eps):
    pos, mass = _rand_system(n, 100 + n)
    a, p = oracle_mod.forces(pos, mass, eps, G=1.3)
    ah, ph = hiprec.forces(pos, mass, eps, G=1.3)
    scale = np.linalg.norm(ah, axis=1, keepdims=True)
    assert np.max(np.abs(a - ah) / scale) <= 1e-14
    assert np.max(np.abs(p - ph) / np.abs(ph)) <= 1e-14


def test_hand_worked_two_body(oracle_mod):
    # particle 1 at (3,4,0) with m=2 seen from the origin: |d| = 5,
    # a_0 = 2 (3,4,0) / 125 = (0.048, 0.064, 0), phi_0 = -2/5.
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    mass = np.array([1.0, 2.0])
    a, p = oracle_mod.forces(pos, mass, 0.0)
    np.testing.assert_allclose(a[0], [0.048, 0.064, 0.0], rtol=1e-15, atol=1e-18)
    np.testing.assert_allclose(a[1], [-0.024, -0.032, 0.0], rtol=1e-15, atol=1e-18)
    np.testing.assert_allclose(p, [-0.4, -0.2], rtol=1e-15)
    # softened: eps = 5 doubles s^2 to 50, s^3 = 50 sqrt(50)
    a, p = oracle_mod.forces(pos, mass, 5.0)
    s3 = 50.0 * math.sqrt(50.0)
    np.testing.assert_allclose(a[0], [6.0 / s3, 8.0 / s3, 0.0], rtol=1e-15)
    np.testing.assert_allclose(p[0], -2.0 / math.sqrt(50.0), rtol=1e-15)


def test_single_particle_and_coincident_pair(oracle_mod):
    a, p = oracle_mod.forces(np.array([[0.3, -0.2, 0.1]]), np.array([2.0]), 0.01)
    assert np.all(a == 0.0) and np.all(p == 0.0)
    pos = np.array([[0.25, 0.5, -1.0], [0.25, 0.5, -1.0]])
    mass = np.array([0.5, 0.75])
    a, p = oracle_mod.forces(pos, mass, 0.01, G=2.0)
    assert np.all(a == 0.0)
    np.testing.assert_allclose(p, [-2.0 * 0.75 / 0.01, -2.0 * 0.5 / 0.01], rtol=1e-15)


def test_newtons_third_law(oracle_mod):
    s = ics.plummer_lognormal(2000, seed=5)
    a, _ = oracle_mod.forces(s.pos, s.mass, 1e-3)
    f = s.mass[:, None] * a
    assert np.abs(f.sum(axis=0)).max() <= 1e-14 * np.abs(f).sum()


def test_translation_invariance(oracle_mod):
    pos, mass = _rand_system(200, 7)
    a0, p0 = oracle_mod.forces(pos, mass, 0.05)
    a1, p1 = oracle_mod.forces(pos + np.array([0.5, -0.25, 0.125]), mass, 0.05)
    np.testing.assert_allclose(a1, a0, rtol=1e-11, atol=1e-11 * np.abs(a0).max())
    np.testing.assert_allclose(p1, p0, rtol=1e-12)


def test_permutation_equivariance(oracle_mod):
    pos, mass = _rand_system(300, 8)
    perm = np.random.default_rng(9).permutation(300)
    a0, p0 = oracle_mod.forces(pos, mass, 0.02)
    a1, p1 = oracle_mod.forces(pos[perm], mass[perm], 0.02)
    np.testing.assert_allclose(a1, a0[perm], rtol=1e-12, atol=1e-12 * np.abs(a0).max())
    np.testing.assert_allclose(p1, p0[perm], rtol=1e-13)


def test_scaling_law(oracle_mod):
    # a(lx; l eps) = a(x; eps) / l^2 and phi -> phi / l; exact for l = 2
    pos, mass = _rand_system(100, 10)
    a0, p0 = oracle_mod.forces(pos, mass, 0.03)
    a2, p2 = oracle_mod.forces(2.0 * pos, mass, 0.06)
    assert np.array_equal(a2, a0 / 4.0) and np.array_equal(p2, p0 / 2.0)
    a3, p3 = oracle_mod.forces(3.0 * pos, mass, 0.09)
    np.testing.assert_allclose(a3, a0 / 9.0, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(p3, p0 / 3.0, rtol=1e-13)
    # G and mass enter linearly
    a4, p4 = oracle_mod.forces(pos, 4.0 * mass, 0.03, G=0.5)
    assert np.array_equal(a4, 2.0 * a0) and np.array_equal(p4, 2.0 * p0)


def test_rows_equal_full_evaluation(oracle_mod):
    s = ics.plummer(1500, seed=2)
    a, p = oracle_mod.forces(s.pos, s.mass, 0.01)
    rows = np.array([0, 17, 1499, 700, 17])
    ar, pr = oracle_mod.forces_rows(s.pos, s.mass, 0.01, rows)
    assert np.array_equal(ar, a[rows]) and np.array_equal(pr, p[rows])


def test_plummer_mean_field(oracle_mod):
    # Continuum Plummer (G = M = a = 1): g(r) = -r / (1 + r^2)^{3/2},
    # Phi(r) = -1 / sqrt(1 + r^2).  Binned sample means must follow them.
    s = ics.plummer(8192, seed=11)
    a, p = oracle_mod.forces(s.pos, s.mass, 1e-3)
    r = np.linalg.norm(s.pos, axis=1)
    ar = (a * s.pos).sum(axis=1) / r
    for lo, hi in [(0.3, 0.6), (0.6, 1.0), (1.0, 1.5), (1.5, 2.5)]:
        sel = (r >= lo) & (r < hi)
        rm = r[sel]
        np.testing.assert_allclose(ar[sel].mean(), (-rm / (1 + rm * rm) ** 1.5).mean(),
                                   rtol=0.05)
        np.testing.assert_allclose(p[sel].mean(), (-1.0 / np.sqrt(1 + rm * rm)).mean(),
                                   rtol=0.03)


def test_stored_50_digit_values(oracle_mod):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "bruteforce_n6.txt")
    rows = np.loadtxt(path)
    a, p = oracle_mod.forces(rows[:, 0:3], rows[:, 3], 0.125)
    scale = np.linalg.norm(rows[:, 4:7], axis=1, keepdims=True)
    assert np.max(np.abs(a - rows[:, 4:7]) / scale) <= 1e-14
    assert np.max(np.abs(p - rows[:, 7]) / np.abs(rows[:, 7])) <= 1e-14
