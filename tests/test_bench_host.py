"""The benchmark's accuracy report on CPU: the per-particle vector-norm
error, the potential error and the component-wise form on a planted case."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_accuracy_on_rows_planted_errors():
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(0)
    ra = rng.normal(size=(1000, 3))
    rp = -0.5 - np.abs(rng.normal(size=1000))
    a = ra.copy()
    p = rp.copy()
    a[17] += 3e-6 * np.linalg.norm(ra[17]) * np.array([0.6, 0.8, 0.0])  # |da| / |a| = 3e-6
    p[5] *= 1 + 2e-6
    r = bench.accuracy_on_rows(a, p, ra, rp)
    assert abs(r["acc_max"] - 3e-6) < 1e-12 and r["acc_median"] == 0.0
    assert abs(r["pot_max"] - 2e-6) < 1e-12 and r["pot_median"] == 0.0
    assert r["pass"]
    # a transposed (x <-> y) result fails the gate
    bad = bench.accuracy_on_rows(a[:, [1, 0, 2]], p, ra, rp)
    assert not bad["pass"] and bad["acc_median"] > 0.1
    # component-wise form: relative to each component
    c = ra.copy()
    c[:, 0] *= 1 + 1e-3
    assert abs(bench.accuracy_on_rows(c, rp, ra, rp)["componentwise_p99"] - 1e-3) < 1e-9
