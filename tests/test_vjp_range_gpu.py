"""The VJP of (a, phi) for a range of rows (one rank's share of a step
adjoint split over GPUs) and the sharded adjoint driver on one rank, against
the whole-system VJP and the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02744_gb300 import binding, ics
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2605_02744_gb300 as pkg
    pkg.build()
    oracle.build()
    binding.lib()


def _full(pos, mass, eps, abar, pbar, o, ws):
    n = mass.shape[0]
    xb = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    mb = torch.empty(n, dtype=torch.float64, device="cuda")
    binding.nb_forces_vjp(pos, mass, eps, abar, pbar, xb, mb, ws, o)
    return host(xb), host(mb)


@pytest.mark.parametrize("prec", ["fp64", "f64acc"])
@pytest.mark.parametrize("n,cuts", [(3001, [0, 1000, 1001, 3001]), (20000, [0, 7000, 13777, 20000])])
def test_rows_equal_the_whole_vjp(prec, n, cuts):
    s = ics.plummer_lognormal(n, seed=8)
    rng = np.random.default_rng(8)
    abar, pbar = rng.normal(size=(n, 3)), rng.normal(size=n)
    pos, mass, ab, pb = dev(s.pos), dev(s.mass), dev(abar), dev(pbar)
    o = binding.make_opts(prec, positions="split")
    ws = binding.workspace(n, 1, o)
    xf, mf = _full(pos, mass, 0.01, ab, pb, o, ws)
    coef = 0.37
    for i0, i1 in zip(cuts[:-1], cuts[1:]):
        xb = torch.full((i1 - i0, 3), 0.25, dtype=torch.float64, device="cuda")
        mb = torch.full((i1 - i0,), -0.5, dtype=torch.float64, device="cuda")
        binding.nb_forces_vjp_range(pos, mass, i0, i1, 0.01, coef, ab, pb, xb, mb, ws, o)
        assert binding.nb_poll_status(ws, o) == binding.NB_OK
        gx, gm = (host(xb) - 0.25) / coef, (host(mb) + 0.5) / coef  # accumulated into
        tol = 1e-12 if prec == "fp64" else 2e-6
        assert np.abs(gx - xf[i0:i1]).max() <= tol * np.abs(xf).max()
        assert np.abs(gm - mf[i0:i1]).max() <= tol * np.abs(mf).max()
    if n <= 3001:
        rx, rm = oracle.forces_vjp(s.pos, s.mass, 0.01, abar, pbar)
        tol = 1e-12 if prec == "fp64" else 2e-6
        assert np.abs(xf - rx).max() <= tol * np.abs(rx).max()
        assert np.abs(mf - rm).max() <= tol * np.abs(rm).max()


def test_bad_ranges_are_refused():
    n = 100
    s = ics.plummer(n, seed=1)
    pos, mass = dev(s.pos), dev(s.mass)
    ab = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    o = binding.make_opts("f64acc")
    ws = binding.workspace(n, 1, o)
    xb = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    mb = torch.zeros(n, dtype=torch.float64, device="cuda")
    for i0, i1 in ((-1, 5), (5, 5), (0, n + 1)):
        with pytest.raises(binding.NbError):
            binding.nb_forces_vjp_range(pos, mass, i0, i1, 0.01, 1.0, ab, None, xb, mb, ws, o)
    with pytest.raises(binding.NbError):
        binding.nb_forces_vjp_range(pos, mass, 0, n, 0.01, float("nan"), ab, None, xb, mb, ws, o)


@pytest.mark.parametrize("prec", ["fp64", "f64acc"])
def test_sharded_adjoint_one_rank_matches_oracle(prec):
    from paper_2605_02744_gb300.sharded import sharded_loss_and_grads
    n, eps, h, steps = 512, 5e-3, 1e-3, 20
    s = ics.plummer(n, seed=0)
    target = ics.perturb_positions(s.pos, 1e-3, seed=2)
    L, xb, vb, mb, (i0, i1) = sharded_loss_and_grads(s.pos, s.vel, s.mass, eps, h, steps, target,
                                                     precision=prec, device="cuda")
    assert (i0, i1) == (0, n)
    rL, gx, gv, gm = oracle.trajectory_loss_grad(s.pos, s.vel, s.mass, eps, h, steps, target)
    g = np.concatenate([host(xb).ravel(), host(vb).ravel(), host(mb)])
    ref = np.concatenate([gx.ravel(), gv.ravel(), gm])
    rel = np.abs(g - ref) / np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max())
    if prec == "fp64":
        assert abs(L - rL) <= 1e-12 * abs(rL)
        assert rel.max() <= 1e-9, rel.max()
    else:
        assert abs(L - rL) <= 1e-6 * abs(rL)
        assert np.median(rel) <= 1e-4 and rel.max() <= 1e-3, (np.median(rel), rel.max())
