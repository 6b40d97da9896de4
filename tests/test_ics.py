"""Pins of the synthetic input generators (Plummer statistics and layouts)."""
import math

import numpy as np
from scipy import stats

from paper_2605_02744_gb300 import ics


def test_plummer_mass_profile_ks():
    s = ics.plummer(20000, seed=0)
    r = np.linalg.norm(s.pos, axis=1)
    # M(<r) = r^3 (1+r^2)^{-3/2}, truncated at X = 0.999
    cdf = lambda x: np.minimum(x ** 3 / (1 + x * x) ** 1.5 / 0.999, 1.0)
    assert stats.kstest(r, cdf).pvalue > 1e-3
    assert r.max() <= 1.0 / math.sqrt(0.999 ** (-2.0 / 3.0) - 1.0) + 1e-6


def test_plummer_energy_and_virial(oracle_mod):
    # Continuum Plummer: E = -3 pi / 64, 2K / |W| = 1 (G = M = a = 1).
    s = ics.plummer(8192, seed=1)
    _, pot = oracle_mod.forces(s.pos, s.mass, 1e-4)
    K, W, E = oracle_mod.energy(s.vel, s.mass, pot)
    assert abs(E - (-3 * math.pi / 64)) < 0.05 * 3 * math.pi / 64
    assert abs(2 * K / abs(W) - 1.0) < 0.05


def test_plummer_velocity_distribution():
    s = ics.plummer(20000, seed=2)
    r = np.linalg.norm(s.pos, axis=1)
    v = np.linalg.norm(s.vel, axis=1)
    q = v / (math.sqrt(2.0) * (1 + r * r) ** -0.25)
    # speeds stay below escape (COM shift aside) and follow g(q) ~ q^2 (1-q^2)^{7/2}
    assert q.max() < 1.05
    grid = np.linspace(0, 1, 2001)
    g = grid ** 2 * (1 - grid ** 2) ** 3.5
    G = np.cumsum(g)
    G /= G[-1]
    assert stats.kstest(np.clip(q, 0, 1), lambda x: np.interp(x, grid, G)).pvalue > 1e-3


def test_plummer_com_frame_and_determinism():
    a = ics.plummer(1000, seed=7)
    b = ics.plummer(1000, seed=7)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.vel, b.vel)
    assert np.abs((a.mass[:, None] * a.pos).sum(0)).max() < 1e-15
    assert np.abs((a.mass[:, None] * a.vel).sum(0)).max() < 1e-15
    assert a.pos.flags["C_CONTIGUOUS"] and a.pos.dtype == np.float64
    assert abs(a.mass.sum() - 1.0) < 1e-14


def test_lognormal_masses():
    s = ics.plummer_lognormal(50000, seed=0)
    assert abs(s.mass.sum() - 1.0) < 1e-12
    assert abs(np.log(s.mass).std() - 0.5) < 0.01
    eq = ics.plummer(50000, seed=0)
    # same phase-space draws up to the mass-weighted COM shift
    d = (s.pos - eq.pos)
    assert np.abs(d - d.mean(0)).max() < 1e-12


def test_batched_layout():
    sizes = ics.batched_sizes()
    assert sizes.shape == (512,) and sizes.min() >= 64 and sizes.max() <= 8192
    # log-uniform: median near sqrt(64 * 8192) = 724
    assert 450 < np.median(sizes) < 1150
    s = ics.batched_plummer(b=6, sizes=np.array([64, 100, 8192, 77, 64, 500]))
    assert list(s.offsets) == [0, 64, 164, 8356, 8433, 8497, 8997]
    for c in range(6):
        lo, hi = s.offsets[c], s.offsets[c + 1]
        assert abs(s.mass[lo:hi].sum() - 1.0) < 1e-12
        assert np.abs((s.mass[lo:hi, None] * s.pos[lo:hi]).sum(0)).max() < 1e-14


def test_perturbation_and_coordinates():
    pos = np.zeros((20000, 3))
    d = ics.perturb_positions(pos, 1e-3, seed=2)
    assert abs(d.std() - 1e-3) < 2e-5
    idx = ics.random_coordinates(16384)
    assert idx.size == 64 and np.unique(idx).size == 64 and idx.max() < 7 * 16384
