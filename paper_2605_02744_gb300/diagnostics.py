"""Post-run diagnostics (host side, not on the hot path).

The paper validates its accelerated runs by comparing the distribution of
per-particle energies after a time t = 3 with the one of its FP64 reference
(Sec. 4.1 and Fig. 4): individual orbits of an N-body system diverge within
a few crossing times, so it is the distribution that two correct runs share.
"""
from __future__ import annotations

import numpy as np


def specific_energies(vel, pot):
    """e_i = |v_i|^2 / 2 + phi_i for every particle (host arrays)."""
    v = np.asarray(vel, dtype=np.float64)
    return 0.5 * (v * v).sum(axis=1) + np.asarray(pot, dtype=np.float64)


def energy_histogram(vel, pot, bins=40, range_=None):
    """(counts, edges) of the specific energies, normalised to a density."""
    e = specific_energies(vel, pot)
    return np.histogram(e, bins=bins, range=range_, density=True)


def compare_distributions(e_a, e_b):
    """Two-sample Kolmogorov-Smirnov statistic and p-value, and the relative
    differences of the mean and the standard deviation."""
    from scipy import stats
    ks = stats.ks_2samp(e_a, e_b)
    return {"ks": float(ks.statistic), "p": float(ks.pvalue),
            "mean_rel": float(abs(e_a.mean() - e_b.mean()) / abs(e_b.mean())),
            "std_rel": float(abs(e_a.std() - e_b.std()) / e_b.std())}
