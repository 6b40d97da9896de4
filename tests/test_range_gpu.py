"""nb_forces_range and nb_kick_drift on the GPU: one system's rows split
into contiguous ranges (the per-rank unit of the multi-GPU split of
Sec. 3.2, approach 1), each evaluated against all N, must together equal
the oracle's forces element by element; and the sharded leapfrog driver on
one rank must reproduce the oracle's KDK steps."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02744_gb300 import binding, ics
from paper_2605_02744_gb300.sharded import ShardedSystem, partition
from tests.gpu_util import TOL, dev, host, rel_err, rel_vec_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2605_02744_gb300 as pkg
    pkg.build()
    oracle.build()
    binding.lib()


@pytest.mark.parametrize("prec", ["kahan", "f64acc", "fp64", "fp32"])
@pytest.mark.parametrize("n,world", [(5000, 2), (20001, 3), (40000, 4), (777, 8), (3, 4)])
def test_ranges_union_matches_oracle(prec, n, world):
    s = ics.plummer_lognormal(n, seed=n + world)
    eps = 0.01
    ra, rp = oracle.forces(s.pos, s.mass, eps)
    pos, mass = dev(s.pos), dev(s.mass)
    o = binding.make_opts(prec, positions="split" if prec == "fp32" else "default")
    ws = binding.workspace(n, 1, o)
    a = np.zeros((n, 3))
    p = np.zeros(n)
    for r in range(world):
        i0, i1, _ = partition(n, world, r)
        if i1 == i0:
            continue
        acc = torch.empty((i1 - i0, 3), dtype=torch.float64, device="cuda")
        pot = torch.empty(i1 - i0, dtype=torch.float64, device="cuda")
        binding.nb_forces_range(pos, mass, i0, i1, eps, acc, pot, ws, o)
        assert binding.nb_poll_status(ws, o) == binding.NB_OK
        a[i0:i1], p[i0:i1] = host(acc), host(pot)
    assert rel_vec_err(a, ra).max() <= TOL[prec] and rel_err(p, rp).max() <= TOL[prec]


def test_range_argument_checks():
    s = ics.plummer(100, seed=1)
    pos, mass = dev(s.pos), dev(s.mass)
    o = binding.make_opts("f64acc")
    ws = binding.workspace(100, 1, o)
    acc = torch.empty((100, 3), dtype=torch.float64, device="cuda")
    for i0, i1 in ((-1, 10), (10, 10), (50, 101), (60, 40)):
        with pytest.raises(binding.NbError) as e:
            binding.nb_forces_range(pos, mass, i0, i1, 0.01, acc, None, ws, o)
        assert e.value.code == binding.NB_ERR_INVALID


def test_kick_drift_matches_definition():
    rng = np.random.default_rng(2)
    x, v, a = rng.normal(size=(3, 1000, 3))
    pos, vel, acc = dev(x), dev(v), dev(a)
    binding.nb_kick_drift(pos, vel, acc, 0.25, 0.5, binding.make_opts("f64acc"))
    torch.cuda.synchronize()
    v1 = v + 0.25 * a
    assert np.abs(host(vel) - v1).max() <= 1e-15 * np.abs(v1).max()
    assert np.abs(host(pos) - (x + 0.5 * v1)).max() <= 1e-15 * np.abs(x + 0.5 * v1).max()


@pytest.mark.parametrize("prec,tol", [("f64acc", 1e-5), ("fp64", 1e-12)])
def test_sharded_driver_one_rank_matches_oracle(prec, tol):
    s = ics.plummer(1024, seed=0)
    eps, h, steps = 0.01, 1e-3, 20
    g = ShardedSystem(s.pos, s.vel, s.mass, eps, precision=prec)
    g.step(h, steps)
    x, v, a = (host(t) for t in g.gather_state())
    e = host(g.energy())
    assert g.ops.poll() == binding.NB_OK
    xo, vo, ao, po = oracle.kdk(s.pos, s.vel, s.mass, eps, h, steps)
    dx = np.abs(xo - s.pos).max()
    assert np.abs(x - xo).max() <= tol * dx
    assert rel_vec_err(a, ao).max() <= tol
    ko, wo, eo = oracle.energy(vo, s.mass, po)
    assert abs(e[2] - eo) <= 10 * tol * abs(eo)
