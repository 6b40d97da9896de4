"""Eq. 1 leaves out j = i exactly in every FP32-pair kernel.

A particle whose own softened term m_i / eps dwarfs its potential makes any
"evaluate the self pair, subtract it afterwards" scheme lose the answer to
FP32 cancellation: here one heavy particle (m = 1) sits among light ones
(m = 1e-6) with eps = 1e-3, so m / eps = 1000 against |phi| ~ 1e-3 -- an
error of ~6e-5 absolute, ~5e-2 relative, if the self term went through an
FP32 sum.  The kernels give that pair a zero mass instead (the tiles that
hold the particle's own slot), so the heavy particle's potential meets the
1e-5 gate like every other particle's.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02744_gb300 import api, binding, ics
from tests.gpu_util import dev, host, rel_err, rel_vec_err

pytestmark = pytest.mark.gpu

EPS = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2605_02744_gb300 as pkg
    pkg.build()
    oracle.build()
    binding.lib()


def heavy_in_light(n, seed, heavy_at=None):
    s = ics.plummer(n, seed=seed)
    mass = np.full(n, 1e-6)
    k = n // 3 if heavy_at is None else heavy_at
    mass[k] = 1.0
    return s.pos, s.vel, mass, k


@pytest.mark.parametrize("prec", ["kahan", "f64acc"])
@pytest.mark.parametrize("pairs,n", [("direct", 3001), ("direct", 70001), ("symmetric", 40001)])
def test_forces_heavy_particle_potential(prec, pairs, n):
    pos, _, mass, k = heavy_in_light(n, 3)
    ra, rp = oracle.forces(pos, mass, EPS) if n < 50000 else \
        oracle.forces_rows(pos, mass, EPS, np.arange(n))
    a, p = api.forces(dev(pos), dev(mass), EPS, precision=prec, pairs=pairs)
    a, p = host(a), host(p)
    assert rel_err(p[k:k + 1], rp[k:k + 1]).max() <= 1e-5, (p[k], rp[k])
    assert rel_vec_err(a, ra).max() <= 1e-5 and rel_err(p, rp).max() <= 1e-5


def test_noalloc_heavy_particle_potential():
    pos, _, mass, k = heavy_in_light(3001, 4)
    ra, rp = oracle.forces(pos, mass, EPS)
    o = binding.make_opts("kahan")
    acc = torch.empty((3001, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(3001, dtype=torch.float64, device="cuda")
    binding.nb_forces_noalloc(dev(pos), dev(mass), EPS, acc, pot, o)
    torch.cuda.synchronize()
    assert rel_err(host(pot), rp).max() <= 1e-5
    assert rel_vec_err(host(acc), ra).max() <= 1e-5


def test_jerk_heavy_particle_potential():
    pos, vel, mass, k = heavy_in_light(3001, 5)
    ra, rj, rp = oracle.forces_jerk(pos, vel, mass, EPS)
    o = binding.make_opts("kahan")
    n = 3001
    acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    jerk = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = binding.workspace(n, 1, o)
    binding.nb_forces_jerk(dev(pos), dev(vel), dev(mass), EPS, acc, jerk, pot, ws, o)
    assert binding.nb_poll_status(ws, o) == binding.NB_OK
    assert rel_err(host(pot), rp).max() <= 1e-5
    assert rel_vec_err(host(acc), ra).max() <= 1e-5


@pytest.mark.parametrize("pairs", ["direct", "symmetric"])
def test_batched_heavy_particle_potential(pairs):
    sizes = [300, 1000, 4097]
    parts = [heavy_in_light(n, 6 + c, heavy_at=(7 * c) % n) for c, n in enumerate(sizes)]
    pos = np.concatenate([p[0] for p in parts])
    mass = np.concatenate([p[2] for p in parts])
    offsets = np.r_[0, np.cumsum(sizes)].astype(np.int64)
    eps_b = np.full(len(sizes), EPS)
    a, p = api.forces_batched(dev(pos), dev(mass), torch.tensor(offsets, device="cuda"),
                              dev(eps_b), precision="kahan", pairs=pairs)
    a, p = host(a), host(p)
    for c in range(len(sizes)):
        lo, hi = offsets[c], offsets[c + 1]
        ra, rp = oracle.forces(pos[lo:hi], mass[lo:hi], EPS)
        assert rel_err(p[lo:hi], rp).max() <= 1e-5, (pairs, c)
        assert rel_vec_err(a[lo:hi], ra).max() <= 1e-5, (pairs, c)
