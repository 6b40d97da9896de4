"""Independent clusters split over ranks by cluster (ShardedBatch), each
rank's share run in this process on one GPU: every cluster's trajectory must
be bit for bit the one of a single run of the whole batch (a cluster's
arithmetic on the batched path does not depend on which other clusters
share its launch), and one cluster is checked against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02744_gb300 import api, ics
from paper_2605_02744_gb300.sharded import ShardedBatch, partition_clusters
from tests.gpu_util import rel_vec_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2605_02744_gb300 as pkg
    pkg.build()
    oracle.build()


@pytest.mark.parametrize("pairs", ["default", "direct"])
def test_cluster_shards_equal_the_whole_batch(pairs):
    sizes = ics.batched_sizes()[:48]
    s = ics.batched_plummer(b=len(sizes), seed=1, sizes=sizes)
    eps = np.full(len(sizes), 0.01)
    steps = 40  # crosses the batched path's re-sort after 32 steps
    full = api.System(s.pos, s.vel, s.mass, eps, offsets=s.offsets, precision="f64acc",
                      pairs=pairs)
    full.step(1e-3, steps)
    assert full.poll() == 0
    fp, fv, fa = (t.cpu().numpy() for t in (full.pos, full.vel, full.acc))
    world = 3
    seen = []
    for r in range(world):
        g = ShardedBatch(s.pos, s.vel, s.mass, s.offsets, eps, world=world, rank=r,
                         device="cuda", pairs=pairs)
        assert g.clusters == partition_clusters(sizes, world)[r]
        g.step(1e-3, steps)  # one call, as the whole batch's (a call starts with a sort)
        rows, p, v, a = g.local_state()
        assert g.ops.poll() == 0
        assert np.array_equal(p.cpu().numpy(), fp[rows])
        assert np.array_equal(v.cpu().numpy(), fv[rows])
        assert np.array_equal(a.cpu().numpy(), fa[rows])
        seen.extend(g.clusters)
    assert sorted(seen) == list(range(len(sizes)))
    # one cluster against the oracle's leapfrog
    c = int(np.argmax(sizes[:8]))
    lo, hi = s.offsets[c], s.offsets[c + 1]
    xo, vo, ao, _ = oracle.kdk(s.pos[lo:hi], s.vel[lo:hi], s.mass[lo:hi], 0.01, 1e-3, steps)
    assert rel_vec_err(fa[lo:hi], ao).max() <= 1e-5
    assert np.abs(fp[lo:hi] - xo).max() <= 1e-8


def test_bench_leg_runs_on_one_rank():
    """bench.py's sharded-batch leg (taken under torchrun with N > 1) on one
    rank: 50 replayed steps of the whole 512-cluster batch."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    r = bench.batched_sharded_rate(torch, 1, torch.device("cuda", 0), None, steps=50)
    assert r["status"] == 0 and r["clusters_on_rank0"] == 512 and r["value"] > 0
