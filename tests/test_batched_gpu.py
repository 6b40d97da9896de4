"""GPU parity of the batched paths (many independent clusters).

Two paths: the default symmetric-pair path (each unordered pair of a cluster
once, warp-granular work items of 2, 4 or 8 j-blocks, per-cluster Hilbert
order) and the persistent
direct-pair kernel (NB_PAIRS_DIRECT, every compiled thread-block-cluster
size).  nb_forces_batched against the oracle cluster by cluster (sizes from
1 to the 8192 maximum), nb_step on a batch against the oracle's leapfrog per
cluster (across a Hilbert re-sort), the 512-cluster workload on a sample of
clusters (smallest and largest included) for 10 steps and on small clusters
for the full 1000 steps with the energy-drift gate, device rejection of an
invalid cluster, bitwise determinism and graph replay.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02744_gb300 import api, binding, ics
from tests.gpu_util import TOL, dev, host, rel_err, rel_vec_err

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 5, 63, 64, 65, 100, 300, 511, 1000, 2049, 8192]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2605_02744_gb300 as pkg
    pkg.build()
    oracle.build()
    binding.lib()


def _batch(sizes, seed=1):
    return ics.batched_plummer(b=len(sizes), seed=seed, sizes=np.array(sizes))


def _eps(b, seed=0):
    return np.random.default_rng(seed).uniform(0.005, 0.02, b)


@pytest.mark.parametrize("prec", ["f64acc", "kahan"])
@pytest.mark.parametrize("tune,pairs", [({"cluster_ctas": c, "threads": t}, "direct")
                                        for t in (256, 512) for c in (2, 4, 8)]
                         + [(None, "symmetric"), ({"item_blocks": 2}, "symmetric"),
                            ({"item_blocks": 4}, "symmetric")])
def test_forces_batched_per_cluster(prec, tune, pairs):
    s = _batch(SIZES)
    eps = _eps(len(SIZES))
    opts = binding.make_opts(prec, tune=tune, pairs=pairs)
    n = s.n
    acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = binding.workspace(n, len(SIZES), opts)
    off = torch.tensor(s.offsets, device="cuda")
    binding.nb_forces_batched(dev(s.pos), dev(s.mass), off, dev(eps), acc, pot, ws, opts)
    assert binding.nb_poll_status(ws, opts) == binding.NB_OK
    a, p = host(acc), host(pot)
    for c in range(len(SIZES)):
        lo, hi = s.offsets[c], s.offsets[c + 1]
        ra, rp = oracle.forces(s.pos[lo:hi], s.mass[lo:hi], eps[c])
        assert rel_vec_err(a[lo:hi], ra).max() <= TOL[prec], (c, SIZES[c])
        assert rel_err(p[lo:hi], rp).max() <= TOL[prec], (c, SIZES[c])


@pytest.mark.parametrize("positions", ["default", "split", "single"])
@pytest.mark.parametrize("pairs", ["default", "direct"])
def test_step_batched_matches_oracle_per_cluster(positions, pairs):
    # 20 steps cross one Hilbert re-sort of every cluster (every 16 steps)
    if positions == "single" and pairs == "direct":
        pytest.skip("the direct batched kernel takes hi/lo or adaptive displacements")
    sizes = [64, 65, 200, 1000, 3000, 7, 1, 8192]
    s = _batch(sizes, seed=3)
    eps = _eps(len(sizes), 1)
    g = api.System(s.pos, s.vel, s.mass, eps, offsets=s.offsets, precision="f64acc",
                   positions=positions, pairs=pairs)
    g.step(1e-3, 20)
    assert g.poll() == binding.NB_OK
    x, v = host(g.pos), host(g.vel)
    for c in range(len(sizes)):
        lo, hi = s.offsets[c], s.offsets[c + 1]
        xo, vo, _, _ = oracle.kdk(s.pos[lo:hi], s.vel[lo:hi], s.mass[lo:hi], eps[c], 1e-3, 20)
        # the force error (<= 1e-5 relative) shows up in the accumulated kicks
        dv = np.abs(vo - s.vel[lo:hi]).max()
        dx = np.abs(xo - s.pos[lo:hi]).max()
        assert np.abs(v[lo:hi] - vo).max() <= 1e-5 * dv + 1e-13, c
        assert np.abs(x[lo:hi] - xo).max() <= 1e-5 * dx + 1e-13, c


def _cluster_energy(x, v, m, pot):
    return 0.5 * (m * (v * v).sum(1)).sum() + 0.5 * (m * pot).sum()


@pytest.mark.parametrize("pairs", ["default", "direct"])
def test_workload_512_clusters_sampled(pairs):
    s = ics.batched_plummer(512, seed=1)
    sizes = np.diff(s.offsets)
    eps = np.full(512, 0.01)
    g = api.System(s.pos, s.vel, s.mass, eps, offsets=s.offsets, precision="f64acc",
                   tune={"cluster_ctas": 8}, pairs=pairs)
    g.step(1e-3, 10)
    assert g.poll() == binding.NB_OK
    x = host(g.pos)
    order = np.argsort(sizes)
    sample = np.unique(np.concatenate([order[:4], order[-4:],
                                       np.random.default_rng(5).choice(512, 8, replace=False)]))
    assert sample.size >= 16 or sample.size == len(set(sample))
    for c in sample:
        lo, hi = s.offsets[c], s.offsets[c + 1]
        xo, _, ao, po = oracle.kdk(s.pos[lo:hi], s.vel[lo:hi], s.mass[lo:hi], 0.01, 1e-3, 10)
        dx = np.abs(xo - s.pos[lo:hi]).max()
        assert np.abs(x[lo:hi] - xo).max() <= 1e-5 * dx + 1e-13, c
        assert rel_vec_err(host(g.acc)[lo:hi], ao).max() <= 1e-5, c
        assert rel_err(host(g.pot)[lo:hi], po).max() <= 1e-5, c


def test_workload_1000_steps_energy_drift_small_clusters():
    s = ics.batched_plummer(512, seed=1)
    sizes = np.diff(s.offsets)
    eps = np.full(512, 0.01)
    g = api.System(s.pos, s.vel, s.mass, eps, offsets=s.offsets, precision="f64acc")
    g.forces()
    pot0 = host(g.pot)
    g.step(1e-3, 1000)
    assert g.poll() == binding.NB_OK
    x1, v1, p1 = host(g.pos), host(g.vel), host(g.pot)
    small = np.where(sizes <= 400)[0][:16]
    assert small.size == 16
    for c in small:
        lo, hi = s.offsets[c], s.offsets[c + 1]
        m = s.mass[lo:hi]
        e0 = _cluster_energy(s.pos[lo:hi], s.vel[lo:hi], m, pot0[lo:hi])
        e1 = _cluster_energy(x1[lo:hi], v1[lo:hi], m, p1[lo:hi])
        xo, vo, _, po = oracle.kdk(s.pos[lo:hi], s.vel[lo:hi], m, 0.01, 1e-3, 1000)
        _, p0r = oracle.forces(s.pos[lo:hi], m, 0.01)
        r0 = oracle.energy(s.vel[lo:hi], m, p0r)[2]
        r1 = oracle.energy(vo, m, po)[2]
        d_ref = abs(r1 - r0) / abs(r0)
        d_gpu = abs(e1 - e0) / abs(e0)
        assert d_gpu <= max(2 * d_ref, d_ref + 1e-6), (c, d_gpu, d_ref)


@pytest.mark.parametrize("pairs", ["default", "direct"])
def test_invalid_cluster_is_rejected_on_device(pairs):
    sizes = [10, 20, 30]
    s = _batch(sizes)
    eps = np.array([0.01, -1.0, 0.01])  # cluster 1 invalid
    opts = binding.make_opts("f64acc", pairs=pairs)
    acc = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    ws = binding.workspace(s.n, 3, opts)
    binding.nb_forces_batched(dev(s.pos), dev(s.mass), torch.tensor(s.offsets, device="cuda"),
                              dev(eps), acc, None, ws, opts)
    assert binding.nb_poll_status(ws, opts) == binding.NB_ERR_INVALID
    a = host(acc)
    assert np.all(a[10:30] == 0.0)  # skipped
    ra, _ = oracle.forces(s.pos[:10], s.mass[:10], 0.01)
    assert rel_vec_err(a[:10], ra).max() <= 1e-5
    assert binding.nb_poll_status(ws, opts) == binding.NB_OK  # cleared


@pytest.mark.parametrize("pairs", ["default", "direct"])
def test_batched_determinism_and_graph_replay(pairs):
    sizes = [500, 64, 2000, 129]
    s = _batch(sizes, seed=9)
    eps = _eps(4, 2)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        a = api.System(s.pos, s.vel, s.mass, eps, offsets=s.offsets, stream=st, pairs=pairs)
        b = api.System(s.pos, s.vel, s.mass, eps, offsets=s.offsets, stream=st, use_graph=True,
                       pairs=pairs)
        for _ in range(2):
            a.step(1e-3, 7)
            b.step(1e-3, 7)
    st.synchronize()
    assert torch.equal(a.pos, b.pos) and torch.equal(a.vel, b.vel) and torch.equal(a.acc, b.acc)


def test_symmetric_and_direct_batched_paths_agree():
    sizes = [8192, 4000, 1, 2, 300, 129, 5000]
    s = _batch(sizes, seed=11)
    eps = _eps(len(sizes), 3)
    out = {}
    for pairs in ("default", "direct"):
        g = api.System(s.pos, s.vel, s.mass, eps, offsets=s.offsets, precision="kahan",
                       pairs=pairs)
        g.step(1e-3, 5)
        assert g.poll() == binding.NB_OK
        out[pairs] = (host(g.pos), host(g.acc), host(g.pot))
    dx = np.abs(out["direct"][0] - s.pos).max()
    assert np.abs(out["default"][0] - out["direct"][0]).max() <= 1e-5 * dx
    assert rel_vec_err(out["default"][1], out["direct"][1]).max() <= 2e-5
    assert rel_err(out["default"][2], out["direct"][2]).max() <= 2e-5


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("f64acc", 1e-5)])
def test_symmetric_batched_policies_and_G(prec, tol):
    # all-FP32 totals (loose gate) and G != 1 on the symmetric batched path
    sizes = [3000, 17, 8192, 640]
    s = _batch(sizes, seed=4)
    eps = _eps(len(sizes), 5)
    G = 0.75
    opts = binding.make_opts(prec, G=G)
    acc = torch.empty((s.n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(s.n, dtype=torch.float64, device="cuda")
    ws = binding.workspace(s.n, len(sizes), opts)
    binding.nb_forces_batched(dev(s.pos), dev(s.mass), torch.tensor(s.offsets, device="cuda"),
                              dev(eps), acc, pot, ws, opts)
    assert binding.nb_poll_status(ws, opts) == binding.NB_OK
    a, p = host(acc), host(pot)
    for c in range(len(sizes)):
        lo, hi = s.offsets[c], s.offsets[c + 1]
        ra, rp = oracle.forces(s.pos[lo:hi], s.mass[lo:hi], eps[c], G)
        assert rel_vec_err(a[lo:hi], ra).max() <= tol, (prec, c)
        assert rel_err(p[lo:hi], rp).max() <= tol, (prec, c)


def test_symmetric_batched_thousands_of_tiny_clusters():
    # 3000 clusters of 1..40 particles: one 128-slot block each, the setup's
    # prefix sums and item order over many systems
    sizes = np.random.default_rng(12).integers(1, 41, 3000)
    s = _batch(list(sizes), seed=13)
    eps = _eps(len(sizes), 7)
    opts = binding.make_opts("kahan")
    acc = torch.empty((s.n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(s.n, dtype=torch.float64, device="cuda")
    ws = binding.workspace(s.n, len(sizes), opts)
    binding.nb_forces_batched(dev(s.pos), dev(s.mass), torch.tensor(s.offsets, device="cuda"),
                              dev(eps), acc, pot, ws, opts)
    assert binding.nb_poll_status(ws, opts) == binding.NB_OK
    a, p = host(acc), host(pot)
    for c in list(range(0, 3000, 97)) + [2999]:
        lo, hi = s.offsets[c], s.offsets[c + 1]
        ra, rp = oracle.forces(s.pos[lo:hi], s.mass[lo:hi], eps[c])
        assert rel_vec_err(a[lo:hi], ra).max() <= 1e-5, c
        assert rel_err(p[lo:hi], rp).max() <= 1e-5, c


@pytest.mark.parametrize("g", [2, 4])
def test_symmetric_batched_item_widths_step(g):
    # narrower work items change only which FP32 sums become FP64 records:
    # 20 steps (one re-sort) against the oracle's leapfrog and the default width
    sizes = [8192, 64, 65, 1000, 3000, 1, 200]
    s = _batch(sizes, seed=21)
    eps = _eps(len(sizes), 8)
    out = {}
    for tune in (None, {"item_blocks": g}):
        sysm = api.System(s.pos, s.vel, s.mass, eps, offsets=s.offsets, precision="f64acc",
                          tune=tune)
        sysm.step(1e-3, 20)
        assert sysm.poll() == binding.NB_OK
        out[g if tune else 8] = (host(sysm.pos), host(sysm.vel), host(sysm.acc))
    x, v, a = out[g]
    for c in range(len(sizes)):
        lo, hi = s.offsets[c], s.offsets[c + 1]
        xo, vo, ao, _ = oracle.kdk(s.pos[lo:hi], s.vel[lo:hi], s.mass[lo:hi], eps[c], 1e-3, 20)
        dv = np.abs(vo - s.vel[lo:hi]).max()
        dx = np.abs(xo - s.pos[lo:hi]).max()
        assert np.abs(v[lo:hi] - vo).max() <= 1e-5 * dv + 1e-13, c
        assert np.abs(x[lo:hi] - xo).max() <= 1e-5 * dx + 1e-13, c
        assert rel_vec_err(a[lo:hi], ao).max() <= 1e-5, c
    assert rel_vec_err(a, out[8][2]).max() <= 2e-5


def test_symmetric_batched_refuses_other_item_widths():
    sizes = [100, 200]
    s = _batch(sizes)
    opts = binding.make_opts("f64acc", tune={"item_blocks": 3})
    acc = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    ws = binding.workspace(s.n, 2, opts)
    with pytest.raises(binding.NbError) as e:
        binding.nb_forces_batched(dev(s.pos), dev(s.mass),
                                  torch.tensor(s.offsets, device="cuda"), dev(_eps(2)), acc,
                                  None, ws, opts)
    assert e.value.code == binding.NB_ERR_INVALID
    assert np.all(host(acc) == 0.0)


@pytest.mark.parametrize("prec,tol", [("kahan", 1e-5), ("fp32", 1e-4)])
def test_symmetric_batched_step_loop_with_G(prec, tol):
    """The fused fold-and-pack of the step loop (merged kicks, G applied
    only when G != 1) under the Kahan and FP32 policies, across a re-sort,
    against the oracle's leapfrog of every cluster with the same G."""
    sizes = [700, 64, 2100, 129]
    s = _batch(sizes, seed=8)
    eps = _eps(len(sizes), 8)
    G, h, steps = 0.75, 1e-3, 40
    g = api.System(s.pos, s.vel, s.mass, eps, offsets=s.offsets, precision=prec, G=G)
    g.step(h, steps)
    assert g.poll() == binding.NB_OK
    x, v, a = host(g.pos), host(g.vel), host(g.acc)
    for c in range(len(sizes)):
        lo, hi = s.offsets[c], s.offsets[c + 1]
        xo, vo, ao, _ = oracle.kdk(s.pos[lo:hi], s.vel[lo:hi], s.mass[lo:hi], eps[c], h, steps, G)
        assert rel_vec_err(a[lo:hi], ao).max() <= tol, (prec, c)
        assert np.abs(x[lo:hi] - xo).max() <= 50 * tol * h * h * steps * np.abs(ao).max(), (prec, c)
        assert np.abs(v[lo:hi] - vo).max() <= 10 * tol * h * steps * np.abs(ao).max(), (prec, c)
