"""Autotuner: cache round trip (CPU) and a tuned choice that is a compiled,
correct shape (GPU)."""
import json

import numpy as np
import pytest


def test_cache_roundtrip(tmp_path, monkeypatch):
    from paper_2605_02744_gb300 import tune as T
    monkeypatch.setenv("NB_TUNE_CACHE", str(tmp_path / "t.json"))
    assert T._bucket(1) == 1 and T._bucket(1000) == 1024 and T._bucket(1 << 20) == 1 << 20
    T._store("dev|sm103|force|kahan|N1024", {"tune": {"threads": 128}, "ms": 1.0})
    T._store("dev|sm103|force|kahan|N2048", {"tune": {"threads": 256}, "ms": 2.0})
    data = json.load(open(tmp_path / "t.json"))
    assert data["dev|sm103|force|kahan|N1024"]["tune"] == {"threads": 128}
    assert len(data) == 2


def test_tie_break_prefers_smaller_resources():
    from paper_2605_02744_gb300 import tune as T
    a = dict(threads=256, i_per_thread=4, tile_j=256, stages=3, ctas_per_sm=2)
    b = dict(threads=128, i_per_thread=2, tile_j=128, stages=3, ctas_per_sm=4)
    assert T._cost(b) < T._cost(a)
    # wider batched items write fewer records
    assert T._cost(dict(item_blocks=8)) < T._cost(dict(item_blocks=2))


def test_batched_path_resolution():
    from paper_2605_02744_gb300 import binding, tune as T
    assert T.batched_pairs("f64acc") == "symmetric"
    assert T.batched_pairs("kahan", "symmetric") == "symmetric"
    assert T.batched_pairs("f64acc", "direct") == "direct"
    assert T.batched_pairs("fp64") == "direct"
    assert all(binding.nb_tune_valid(c) for c in T.BATCHED_SYM_CANDIDATES)


@pytest.mark.gpu
def test_autotune_forces_picks_a_correct_compiled_shape(tmp_path, monkeypatch):
    import torch

    import oracle
    from paper_2605_02744_gb300 import api, binding, ics, tune as T
    from tests.gpu_util import rel_vec_err
    monkeypatch.setenv("NB_TUNE_CACHE", str(tmp_path / "t.json"))
    s = ics.plummer(20000, seed=1)
    pos, mass = torch.tensor(s.pos, device="cuda"), torch.tensor(s.mass, device="cuda")
    best = T.autotune_forces(pos, mass, 0.01, "kahan", reps=2)
    assert binding.nb_tune_valid(best)
    assert T.lookup("force", "kahan", 20000) == best
    a, _ = api.forces(pos, mass, 0.01, precision="kahan", tune="auto")
    ra, _ = oracle.forces_rows(s.pos, s.mass, 0.01, np.arange(0, 20000, 97))
    assert rel_vec_err(a.cpu().numpy()[::97], ra).max() <= 1e-5


@pytest.mark.gpu
def test_autotune_batched(tmp_path, monkeypatch):
    import torch

    from paper_2605_02744_gb300 import ics, tune as T
    monkeypatch.setenv("NB_TUNE_CACHE", str(tmp_path / "t.json"))
    s = ics.batched_plummer(b=24, seed=1)
    args = (torch.tensor(s.pos, device="cuda"), torch.tensor(s.vel, device="cuda"),
            torch.tensor(s.mass, device="cuda"), s.offsets, np.full(24, 0.01), 1e-3)
    x0 = args[0].clone()
    best = T.autotune_batched(*args, nsteps=5, reps=2, pairs="direct")
    assert torch.equal(args[0], x0)  # trial runs step copies
    assert best["cluster_ctas"] in (2, 4, 8)
    assert T.lookup("batched-direct", "f64acc", s.n) == best
    # the default (symmetric) path tunes its work-item width
    best = T.autotune_batched(*args, nsteps=5, reps=2)
    assert best["item_blocks"] in (2, 4, 8)
    assert T.lookup("batched-symmetric", "f64acc", s.n) == best


@pytest.mark.gpu
def test_batched_auto_tune_matches_the_oracle(tmp_path, monkeypatch):
    import torch

    import oracle
    from paper_2605_02744_gb300 import api, ics
    from tests.gpu_util import rel_vec_err
    monkeypatch.setenv("NB_TUNE_CACHE", str(tmp_path / "t.json"))
    s = ics.batched_plummer(b=12, seed=3)
    eps = np.full(12, 0.01)
    sysm = api.System(s.pos, s.vel, s.mass, eps, offsets=s.offsets, tune="auto")
    assert sysm.opts.tune.contents.item_blocks in (2, 4, 8)
    sysm.forces()
    assert sysm.poll() == 0
    a = sysm.acc.cpu().numpy()
    for c in range(12):
        o0, o1 = s.offsets[c], s.offsets[c + 1]
        ra, _ = oracle.forces(s.pos[o0:o1], s.mass[o0:o1], eps[c])
        assert rel_vec_err(a[o0:o1], ra).max() <= 1e-5
