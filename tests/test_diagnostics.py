import numpy as np

from paper_2605_02744_gb300 import diagnostics


def test_specific_energy_and_histogram():
    vel = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    pot = np.array([-1.0, -0.5])
    np.testing.assert_allclose(diagnostics.specific_energies(vel, pot), [-0.5, 1.5])
    counts, edges = diagnostics.energy_histogram(vel, pot, bins=2, range_=(-1.0, 2.0))
    assert edges.shape == (3,) and abs((counts * np.diff(edges)).sum() - 1.0) < 1e-12


def test_compare_identical_and_shifted():
    rng = np.random.default_rng(0)
    a = rng.normal(-0.5, 0.1, 5000)
    same = diagnostics.compare_distributions(a, a.copy())
    assert same["ks"] == 0.0 and same["p"] == 1.0
    shifted = diagnostics.compare_distributions(a + 0.05, a)
    assert shifted["p"] < 1e-6
