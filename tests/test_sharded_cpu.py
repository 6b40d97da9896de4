"""The multi-rank split of one system (paper_2605_02744_gb300.sharded) on
CPU ranks over gloo: the contiguous partition, the order of the position
all-gather and the reassembly of the rows, driven through the same
ShardedSystem the GPU path uses, with a stand-in for the library's kernels
(the oracle's exact rows and the KDK kick / drift in float64).  World sizes
2 and 3 (ragged last rank) must reproduce the oracle's single-process
leapfrog."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_covers_every_row_once():
    from paper_2605_02744_gb300.sharded import partition
    for n in (1, 2, 7, 100, 1001, 4096):
        for world in (1, 2, 3, 4, 8):
            rows = []
            for r in range(world):
                i0, i1, c = partition(n, world, r)
                assert c == -(-n // world)
                assert i1 - i0 <= c and 0 <= i0 <= i1 <= n
                assert i0 == min(r * c, n)
                rows.extend(range(i0, i1))
            assert rows == list(range(n))
    with pytest.raises(ValueError):
        partition(10, 2, 2)


class OracleOps:
    """CPU stand-in for the library's kernels (test infrastructure only)."""

    def forces_range(self, pos_all, mass_all, eps, i0, i1, acc, pot):
        import oracle
        a, p = oracle.forces_rows(pos_all.numpy(), mass_all.numpy(), eps, np.arange(i0, i1))
        acc.copy_(torch.from_numpy(a))
        pot.copy_(torch.from_numpy(p))

    def kick_drift(self, pos, vel, acc, kick, drift):
        vel.copy_(vel + kick * acc)
        if drift != 0.0:
            pos.copy_(pos + drift * vel)

    def energy_rows(self, pos, vel, acc, mass, pot):
        k = 0.5 * (mass[:, None] * vel * vel).sum()
        w = 0.5 * (mass * pot).sum()
        return torch.stack([k, w])

    def vjp_range(self, pos_all, mass_all, eps, i0, i1, coef, abar_all, pos_bar, mass_bar):
        import oracle
        xb, mb = oracle.forces_vjp(pos_all.numpy(), mass_all.numpy(), eps,
                                   coef * abar_all.numpy())
        pos_bar.add_(torch.from_numpy(xb[i0:i1]))
        mass_bar.add_(torch.from_numpy(mb[i0:i1]))

    def kick(self, vel, acc, kick):
        vel.copy_(vel + kick * acc)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2605_02744_gb300 import ics
    from paper_2605_02744_gb300.sharded import ShardedSystem
    oracle.build()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = ics.plummer(301, seed=9)
        g = ShardedSystem(s.pos, s.vel, s.mass, 0.02, ops=OracleOps(), device="cpu")
        g.step(1e-3, 5)
        pos, vel, acc = g.gather_state()
        e = g.energy()
        out.put((rank, g.i0, g.i1, pos.numpy(), vel.numpy(), acc.numpy(), e.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_leapfrog_gloo_matches_oracle(world, oracle_mod):
    from paper_2605_02744_gb300 import ics
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = ics.plummer(301, seed=9)
    xo, vo, ao, po = oracle_mod.kdk(s.pos, s.vel, s.mass, 0.02, 1e-3, 5)
    ko, wo, eo = oracle_mod.energy(vo, s.mass, po)
    # the ranks' rows tile 0..N-1 in order, and every rank reassembles the same state
    assert [r[1] for r in res] == [min(k * -(-301 // world), 301) for k in range(world)]
    assert res[-1][2] == 301
    for r in res:
        assert np.abs(r[3] - xo).max() <= 1e-13 and np.abs(r[4] - vo).max() <= 1e-13
        assert np.abs(r[5] - ao).max() <= 1e-12 * np.abs(ao).max()
        assert np.allclose(r[6], [ko, wo, eo], rtol=1e-12, atol=0.0)


# ---------------------------------------------------------------- by cluster
def test_partition_clusters_covers_each_cluster_once_and_balances():
    from paper_2605_02744_gb300 import ics
    from paper_2605_02744_gb300.sharded import partition_clusters
    for sizes in ([5], [3, 9, 1, 7, 7, 2], list(ics.batched_sizes())):
        for world in (1, 2, 3, 8, 600):
            parts = partition_clusters(sizes, world)
            assert len(parts) == world
            assert sorted(c for p in parts for c in p) == list(range(len(sizes)))
            assert all(p == sorted(p) for p in parts)
            loads = [sum(sizes[c] ** 2 for c in p) for p in parts]
            # greedy largest-first: no rank exceeds the mean by more than one cluster
            assert max(loads) <= sum(loads) / world + max(sizes) ** 2
    with pytest.raises(ValueError):
        partition_clusters([1, 2], 0)


class OracleBatchOps:
    """CPU stand-in for the batched path: the oracle's leapfrog per cluster
    (test infrastructure only)."""

    def bind(self, pos, vel, mass, offsets, eps):
        self.off, self.eps, self.mass = offsets, eps, mass
        self.pos, self.vel = pos.copy(), vel.copy()
        self.acc = np.zeros_like(pos)
        self.pot = np.zeros(mass.shape[0])
        self.valid = False

    def step(self, dt, nsteps):
        import oracle
        for c in range(len(self.eps)):
            lo, hi = self.off[c], self.off[c + 1]
            x, v, a, p = oracle.kdk(self.pos[lo:hi], self.vel[lo:hi], self.mass[lo:hi],
                                    self.eps[c], dt, nsteps,
                                    acc=self.acc[lo:hi] if self.valid else None)
            self.pos[lo:hi], self.vel[lo:hi], self.acc[lo:hi], self.pot[lo:hi] = x, v, a, p
        self.valid = True

    def energy_kw(self):
        k = 0.5 * (self.mass[:, None] * self.vel ** 2).sum()
        w = 0.5 * (self.mass * self.pot).sum()
        return torch.tensor([k, w], dtype=torch.float64)

    def state(self):
        return tuple(torch.from_numpy(a) for a in (self.pos, self.vel, self.acc))


BATCH_SIZES = [50, 120, 33, 80, 64, 10, 90]


def _batch_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2605_02744_gb300 import ics
    from paper_2605_02744_gb300.sharded import ShardedBatch
    oracle.build()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = ics.batched_plummer(b=len(BATCH_SIZES), seed=3, sizes=BATCH_SIZES)
        eps = np.linspace(0.01, 0.03, len(BATCH_SIZES))
        g = ShardedBatch(s.pos, s.vel, s.mass, s.offsets, eps, ops=OracleBatchOps(), device="cpu")
        g.step(1e-3, 3)
        g.step(1e-3, 2)
        pos, vel, acc = g.gather_state()
        e = g.energy()
        out.put((rank, g.clusters, pos, vel, acc, e.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_batch_gloo_matches_single_process(world, oracle_mod):
    from paper_2605_02744_gb300 import ics
    from paper_2605_02744_gb300.sharded import partition_clusters
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_batch_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = ics.batched_plummer(b=len(BATCH_SIZES), seed=3, sizes=BATCH_SIZES)
    eps = np.linspace(0.01, 0.03, len(BATCH_SIZES))
    xo, vo, ao = np.zeros_like(s.pos), np.zeros_like(s.pos), np.zeros_like(s.pos)
    k = w = 0.0
    for c in range(len(BATCH_SIZES)):
        lo, hi = s.offsets[c], s.offsets[c + 1]
        x, v, a, p = oracle_mod.kdk(s.pos[lo:hi], s.vel[lo:hi], s.mass[lo:hi], eps[c], 1e-3, 3)
        x, v, a, p = oracle_mod.kdk(x, v, s.mass[lo:hi], eps[c], 1e-3, 2, acc=a)
        xo[lo:hi], vo[lo:hi], ao[lo:hi] = x, v, a
        k += 0.5 * (s.mass[lo:hi, None] * v ** 2).sum()
        w += 0.5 * (s.mass[lo:hi] * p).sum()
    parts = partition_clusters(BATCH_SIZES, world)
    for r in res:
        assert r[1] == parts[r[0]]
        # every rank reassembles the whole batch, equal to the single-process run
        assert np.array_equal(r[2], xo) and np.array_equal(r[3], vo) and np.array_equal(r[4], ao)
        assert np.allclose(r[5], [k, w, k + w], rtol=1e-13, atol=0.0)


# ------------------------------------------------------------ the adjoint
def _adjoint_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2605_02744_gb300 import ics
    from paper_2605_02744_gb300.sharded import sharded_loss_and_grads
    oracle.build()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = ics.plummer(N_ADJ[world], seed=4)
        target = s.pos + 0.01
        L, xb, vb, mb, (i0, i1) = sharded_loss_and_grads(
            s.pos, s.vel, s.mass, 0.05, 1e-3, 6, target, ops=OracleOps(), device="cpu")
        out.put((rank, L, i0, i1, xb.numpy(), vb.numpy(), mb.numpy()))
    finally:
        dist.destroy_process_group()


N_ADJ = {2: 97, 3: 97, 4: 5}  # 5 particles on 4 ranks: rows 2, 2, 1, 0


@pytest.mark.parametrize("world", [2, 3, 4])
def test_sharded_adjoint_gloo_matches_oracle(world, oracle_mod):
    """Two cotangent all-gathers per step and the rows' VJPs reproduce the
    oracle's unmerged trajectory adjoint, row by row (also with a rank that
    owns no rows and only takes part in the gathers)."""
    from paper_2605_02744_gb300 import ics
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_adjoint_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n = N_ADJ[world]
    s = ics.plummer(n, seed=4)
    L, gx, gv, gm = oracle_mod.trajectory_loss_grad(s.pos, s.vel, s.mass, 0.05, 1e-3, 6,
                                                    s.pos + 0.01)
    for rank, Lr, i0, i1, xb, vb, mb in res:
        assert abs(Lr - L) <= 1e-14 * abs(L)
        assert xb.shape == (i1 - i0, 3) and mb.shape == (i1 - i0,)
        if i1 == i0:
            continue
        scale = np.abs(np.concatenate([gx.ravel(), gv.ravel()])).max()
        assert np.abs(xb - gx[i0:i1]).max() <= 1e-13 * scale
        assert np.abs(vb - gv[i0:i1]).max() <= 1e-13 * scale
        assert np.abs(mb - gm[i0:i1]).max() <= 1e-13 * np.abs(gm).max()
    assert res[-1][3] == n


def test_sharded_batch_rank_without_clusters():
    """More ranks than clusters: the idle rank steps nothing and reports
    zeros."""
    from paper_2605_02744_gb300 import ics
    from paper_2605_02744_gb300.sharded import ShardedBatch
    s = ics.batched_plummer(b=3, seed=3, sizes=[20, 30, 40])
    g = ShardedBatch(s.pos, s.vel, s.mass, s.offsets, 0.02, ops=OracleBatchOps(), world=5,
                     rank=4, device="cpu")
    assert g.clusters == [] and g.ops is None and g.rows.size == 0
    g.step(1e-3, 3)
    assert g.energy().tolist() == [0.0, 0.0, 0.0]
    rows, p, v, a = g.local_state()
    assert rows.size == 0 and p.shape == (0, 3)
    busy = ShardedBatch(s.pos, s.vel, s.mass, s.offsets, 0.02, ops=OracleBatchOps(), world=5,
                        rank=0, device="cpu")
    assert busy.clusters == [2]
