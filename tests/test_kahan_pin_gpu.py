"""The Kahan-compensated accumulation is live: an input where plain FP32
running totals lose part of the answer and compensated ones keep it.

The paper computes its pair terms in FP32 on the device (Sec. 3.1); how a
particle's FP32 partial sums (one per j-tile, or per flush of the register
sums) are then combined is the accumulation policy.  The input makes that
combination decide the result for one particle, the target (particle 0,
at the origin):

* particle 1, first in order after the target, pulls it with |a| ~ 1.5, so
  the target's running total sits in [1, 2) from the first partial on;
* the other 2^20 - 2 particles lie on a spherical cap of radius 30 around
  +x; each pulls the target by at most 2.2e-10, so a partial sum of up to
  256 of them stays below half a unit in the last place of the running total
  (5.96e-8) and is rounded away entirely by a plain FP32 add -- 2^20 of them
  add up to ~2.1e-4, i.e. a relative error of ~1.4e-4 in the target's
  acceleration (14 times the 1e-5 gate) for plain FP32 totals, while a
  Kahan (or an FP64) total keeps them.

This is the textbook contrast between recursive summation (error growing
with the number of terms) and compensated summation (error ~2u independent
of it), with no cancellation involved.  Displacements are split hi/lo
(positions="split") so that rounding of the positions plays no part.  Both
FP32-pair kernel families are checked: the direct kernel with 64-particle
j-tiles, and the symmetric kernel, whose register sums (two streams of 128
terms) are added and flushed into the policy every 256 pair terms.
"""
import numpy as np
import pytest

N = 1 << 20
EPS = 0.01
HEAVY = 1.5
R_CAP = 30.0
Q_MAX = 2.2e-10  # largest pull of one light particle on the target


def cap_input(n=N, seed=11):
    rng = np.random.default_rng(seed)
    pos = np.zeros((n, 3))
    mass = np.zeros(n)
    pos[1] = (1.0, 0.0, 0.0)
    mass[1] = HEAVY
    k = n - 2
    # uniform on the cap of half-angle 30 degrees around +x
    cz = rng.uniform(np.cos(np.pi / 6), 1.0, size=k)
    ph = rng.uniform(0.0, 2 * np.pi, size=k)
    sz = np.sqrt(1.0 - cz ** 2)
    pos[2:] = R_CAP * np.stack([cz, sz * np.cos(ph), sz * np.sin(ph)], axis=1)
    mass[2:] = Q_MAX * (R_CAP ** 2 + EPS ** 2) ** 1.5 / R_CAP
    return pos, mass


def _target_terms(pos, mass):
    d = pos - pos[0]
    r2 = (d ** 2).sum(1) + EPS ** 2
    t = (mass / r2 ** 1.5) * d[:, 0]
    t[0] = 0.0
    return t


@pytest.mark.parametrize("group", [64, 256])
def test_input_defeats_plain_fp32_totals_but_not_kahan(group):
    """CPU emulation of the policy step (FP32 partial sums of `group` terms
    in particle order, then an FP32 running total, plain or Kahan): the
    premise of the GPU test below."""
    pos, mass = cap_input()
    t = _target_terms(pos, mass)
    assert np.abs(t[2:]).max() <= Q_MAX * 1.0001
    exact = t.sum()
    parts = t.astype(np.float32).reshape(-1, group).sum(axis=1, dtype=np.float32)
    plain = np.float32(0.0)
    ks, kc = np.float32(0.0), np.float32(0.0)
    for g in parts:
        plain = np.float32(plain + g)
        y = np.float32(g - kc)
        tt = np.float32(ks + y)
        kc = np.float32(np.float32(tt - ks) - y)
        ks = tt
    kahan = float(ks) - float(kc)
    assert abs(kahan - exact) / abs(exact) < 1e-6
    assert abs(float(plain) - exact) / abs(exact) > 1e-4


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("pairs", ["direct", "symmetric"])
def test_kahan_keeps_what_fp32_loses(pairs):
    import torch

    import oracle
    import paper_2605_02744_gb300 as pkg
    from paper_2605_02744_gb300 import api
    from tests.gpu_util import dev, host, rel_err, rel_vec_err
    pkg.build()
    oracle.build()
    pos, mass = cap_input()
    rows = np.r_[0, 1, np.random.default_rng(12).choice(np.arange(2, N), 62, replace=False)]
    ra, rp = oracle.forces_rows(pos, mass, EPS, rows)
    tune = {"threads": 128, "i_per_thread": 1, "tile_j": 64, "stages": 2} \
        if pairs == "direct" else None
    err = {}
    for prec in ("fp32", "kahan", "f64acc"):
        a, p = api.forces(dev(pos), dev(mass), EPS, precision=prec, positions="split",
                          pairs=pairs, tune=tune)
        torch.cuda.synchronize()
        a, p = host(a)[rows], host(p)[rows]
        e = rel_vec_err(a, ra)
        err[prec] = e[0]
        if prec != "fp32":
            # the compensated policies meet the gate on every sampled row
            assert e.max() <= 1e-5 and rel_err(p, rp).max() <= 1e-5, (pairs, prec, e.max())
    # the target: compensated totals keep the light pieces ...
    assert err["kahan"] <= 1e-6 and err["f64acc"] <= 1e-6, (pairs, err)
    # ... which plain FP32 totals round away (expected ~1.4e-4)
    assert err["fp32"] > 1e-4, (pairs, err)
