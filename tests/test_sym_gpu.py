"""GPU parity of the symmetric-pair path (NB_PAIRS_SYMMETRIC) with the oracle.

Each unordered pair is evaluated once and applied to both particles (Eq. 1
changes sign under i <-> j apart from the masses).  Covered: 1, 2, 3 and 17
row blocks of 2048 slots with ragged last blocks, the three displacement
modes and three FP32-pair policies, the fixed-point combination of j-side
partials and row totals across CTAs, the fused closing half-kick of a step
loop (and the Hilbert order kept across steps), G scaling, a missing
potential output, run-to-run bitwise determinism, agreement with the direct
path, a 2^22 + 777-particle evaluation on sampled rows, a small softening
length (the fixed-point grid against the FP64 gate), the host-side refusals
(eps = 0, a workspace sized for the direct path) and the kernel timer past
its 64 event pairs.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02744_gb300 import api, binding, ics
from tests.gpu_util import dev, host, rel_err, rel_vec_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2605_02744_gb300 as pkg
    pkg.build()
    oracle.build()
    binding.lib()


def _system(n, seed):
    if n == 1:
        return ics.ParticleSet(np.array([[0.3, -0.2, 0.1]]), np.zeros((1, 3)), np.array([0.7]))
    return ics.plummer_lognormal(n, seed=seed)


def _forces(s, eps, prec, positions="default", pairs="symmetric", G=1.0, with_pot=True):
    a, p = api.forces(dev(s.pos), dev(s.mass), eps, precision=prec, G=G, with_pot=with_pot,
                      positions=positions, pairs=pairs)
    return host(a), (host(p) if with_pot else None)


@pytest.mark.parametrize("n", [1, 2, 100, 2048, 2049, 5000, 6144, 34000])
@pytest.mark.parametrize("positions", ["split", "adaptive", "single"])
def test_symmetric_matches_oracle(n, positions):
    s = _system(n, n)
    eps = 0.01 if n < 30000 else 2e-3
    ra, rp = oracle.forces(s.pos, s.mass, eps)
    for prec in ("kahan", "f64acc", "fp32"):
        a, p = _forces(s, eps, prec, positions)
        ea, ep = rel_vec_err(a, ra).max(), rel_err(p, rp).max()
        if prec == "fp32" or positions == "single":
            # single-float displacements and FP32 totals: no better than the
            # direct kernel with the same options, up to summation order
            da, dp = _forces(s, eps, prec, positions, pairs="direct")
            tol_a = max(2 * rel_vec_err(da, ra).max(), 1e-5)
            tol_p = max(2 * rel_err(dp, rp).max(), 1e-5)
            assert ea <= tol_a and ep <= tol_p, (prec, positions, n, ea, ep, tol_a, tol_p)
        else:
            assert ea <= 1e-5 and ep <= 1e-5, (prec, positions, n, ea, ep)


def test_single_particle_is_exactly_zero():
    s = _system(1, 0)
    for prec in ("kahan", "f64acc", "fp32"):
        a, p = _forces(s, 0.05, prec)
        assert np.all(a == 0.0) and np.all(p == 0.0)


def test_gravitational_constant_and_no_potential():
    s = _system(5000, 2)
    ra, rp = oracle.forces(s.pos, s.mass, 0.01, 2.5)
    a, p = _forces(s, 0.01, "f64acc", G=2.5)
    assert rel_vec_err(a, ra).max() <= 1e-5 and rel_err(p, rp).max() <= 1e-5
    a2, _ = _forces(s, 0.01, "f64acc", G=2.5, with_pot=False)
    assert np.array_equal(a, a2)


def test_bitwise_determinism_and_direct_agreement():
    s = ics.plummer(70000, seed=3)
    outs = [api.forces(dev(s.pos), dev(s.mass), 1e-3, precision="kahan") for _ in range(2)]
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    d = api.forces(dev(s.pos), dev(s.mass), 1e-3, precision="kahan", pairs="direct")
    assert rel_vec_err(host(outs[0][0]), host(d[0])).max() <= 1e-5
    assert rel_err(host(outs[0][1]), host(d[1])).max() <= 1e-5


@pytest.mark.parametrize("n,steps", [(5000, 12), (40000, 20)])
def test_step_loop_matches_oracle(n, steps):
    # the closing half-kick is fused into the fold; 40000 particles step on
    # the Hilbert-sorted pack, re-sorted every 16 steps
    s = ics.plummer(n, seed=7)
    eps, h = 2e-3, 1e-4
    g = api.System(s.pos, s.vel, s.mass, eps, precision="f64acc", pairs="symmetric")
    g.step(h, steps)
    assert g.poll() == binding.NB_OK
    if n <= 5000:
        xo, vo, ao, _ = oracle.kdk(s.pos, s.vel, s.mass, eps, h, steps)
        dx = np.abs(xo - s.pos).max()
        dv = np.abs(vo - s.vel).max()
        assert np.abs(host(g.pos) - xo).max() <= 1e-5 * dx
        assert np.abs(host(g.vel) - vo).max() <= 1e-5 * dv
        assert rel_vec_err(host(g.acc), ao).max() <= 1e-5
    else:
        b = api.System(s.pos, s.vel, s.mass, eps, precision="f64acc", pairs="direct")
        b.step(h, steps)
        dx = np.abs(host(b.pos) - s.pos).max()
        assert rel_vec_err(host(g.acc), host(b.acc)).max() <= 2e-5
        assert np.abs(host(g.pos) - host(b.pos)).max() <= 1e-6 * dx


def test_refusals():
    s = _system(3000, 5)
    o = binding.make_opts("f64acc", pairs="symmetric")
    acc = torch.empty((s.n, 3), dtype=torch.float64, device="cuda")
    ws = binding.workspace(s.n, 1, o)
    with pytest.raises(binding.NbError) as e:
        binding.nb_forces(dev(s.pos), dev(s.mass), 0.0, acc, None, ws, o)
    assert e.value.code == binding.NB_ERR_UNSUPPORTED
    small = binding.workspace(s.n, 1, binding.make_opts("f64acc", pairs="direct"))
    with pytest.raises(binding.NbError) as e:
        binding.nb_forces(dev(s.pos), dev(s.mass), 0.01, acc, None, small, o)
    assert e.value.code == binding.NB_ERR_WORKSPACE
    # default pairs with eps = 0 take the guarded direct kernel
    a, p = _forces(s, 0.0, "f64acc", pairs="default")
    ra, rp = oracle.forces(s.pos, s.mass, 0.0)
    assert rel_vec_err(a, ra).max() <= 1e-5


@pytest.mark.slow
def test_four_million_particles_sampled_rows():
    # 2^22 + 777 particles: 2049 row blocks with a ragged last one (scratch
    # O(N): 64 B per particle of fixed-point totals)
    n = (1 << 22) + 777
    s = ics.plummer(n, seed=22)
    r = np.linalg.norm(s.pos, axis=1)
    order = np.argsort(r)
    rows = np.unique(np.concatenate([np.random.default_rng(8).choice(n, 400, replace=False),
                                     order[:32], order[-32:], np.arange(n - 40, n)]))
    o = binding.make_opts("kahan")
    assert binding.nb_workspace_bytes(n, 1, o) <= 2 << 30
    acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = binding.workspace(n, 1, o)
    binding.nb_forces(dev(s.pos), dev(s.mass), 1e-3, acc, pot, ws, o)
    assert binding.nb_poll_status(ws, o) == binding.NB_OK
    ra, rp = oracle.forces_rows(s.pos, s.mass, 1e-3, rows)
    assert rel_vec_err(host(acc)[rows], ra).max() <= 1e-5
    assert rel_err(host(pot)[rows], rp).max() <= 1e-5
    del ws


def test_small_softening_fixed_point_grid():
    # eps = 1e-6 raises the a-priori bound that fixes the fixed-point grid
    # (N max|m| 0.385 / eps^2); FP64 pairs still meet the FP64 gate
    s = _system(40000, 9)
    ra, rp = oracle.forces(s.pos, s.mass, 1e-6)
    a, p = _forces(s, 1e-6, "fp64")
    assert rel_vec_err(a, ra).max() <= 1e-12 and rel_err(p, rp).max() <= 1e-12
    a1, p1 = _forces(s, 1e-6, "fp64")
    assert np.array_equal(a, a1) and np.array_equal(p, p1)


@pytest.mark.parametrize("n", [1, 2, 100, 2049, 5000, 34000])
def test_symmetric_fp64_matches_oracle(n):
    # FP64 pairs and sums with each unordered pair once: the FP64 gate
    s = _system(n, n + 1)
    eps = 0.01 if n < 30000 else 2e-3
    ra, rp = oracle.forces(s.pos, s.mass, eps)
    a, p = _forces(s, eps, "fp64")
    assert rel_vec_err(a, ra).max() <= 1e-12 and rel_err(p, rp).max() <= 1e-12
    d, dp = _forces(s, eps, "fp64", pairs="direct")
    assert rel_vec_err(a, d).max() <= 1e-12


def test_symmetric_fp64_step_loop():
    s = ics.plummer_lognormal(40000, seed=17)
    eps, h, steps = 1e-3, 1e-4, 5
    g = api.System(s.pos, s.vel, s.mass, eps, precision="fp64")  # default: symmetric
    b = api.System(s.pos, s.vel, s.mass, eps, precision="fp64", pairs="direct")
    g.step(h, steps)
    b.step(h, steps)
    assert g.poll() == binding.NB_OK
    dx = np.abs(host(b.pos) - s.pos).max()
    assert np.abs(host(g.pos) - host(b.pos)).max() <= 1e-12 * max(dx, 1.0)
    assert rel_vec_err(host(g.acc), host(b.acc)).max() <= 1e-12
    assert rel_err(host(g.pot), host(b.pot)).max() <= 1e-12


def test_kernel_timing_hook_times_each_pair_launch():
    # nb_kernel_timing: one event pair per symmetric pair-kernel launch, on
    # the launch stream; the pair kernel is part of each call's time
    s = _system(40000, 3)
    pos, mass = dev(s.pos), dev(s.mass)
    api.forces(pos, mass, 1e-3, precision="kahan")  # warm-up (graph of sizes, opt-ins)
    torch.cuda.synchronize()
    binding.nb_kernel_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        api.forces(pos, mass, 1e-3, precision="kahan")
    e1.record()
    torch.cuda.synchronize()
    ms, n = binding.nb_kernel_time()
    binding.nb_kernel_timing(False)
    assert n == 3
    assert 0.0 < ms <= e0.elapsed_time(e1)
    # stopped: further launches are not recorded, and the record stays
    api.forces(pos, mass, 1e-3, precision="kahan")
    torch.cuda.synchronize()
    assert binding.nb_kernel_time()[1] == 3
    # more launches than the ring's 64 event pairs: the oldest are folded in
    binding.nb_kernel_timing(True)
    for _ in range(70):
        api.forces(pos, mass, 1e-3, precision="kahan")
    ms70, n70 = binding.nb_kernel_time()
    binding.nb_kernel_timing(False)
    assert n70 == 70 and ms70 > 10 * ms / 3
