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
