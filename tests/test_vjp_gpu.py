"""GPU parity of the force VJP and of the leapfrog adjoint.

nb_forces_vjp against the oracle's block-by-block Jacobian product (with and
without a potential cotangent, eps > 0 and the guarded eps = 0 kernel, FP32
and FP64 pairs); the trajectory gradient of a final-position loss against
the oracle's unmerged step adjoint; the time-reversed and recomputed
backward passes against each other.  The 16384-particle, 200-step adjoint
workload is checked against the oracle in test_adjoint_c4_gpu.py.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02744_gb300 import adjoint, binding, ics
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2605_02744_gb300 as pkg
    pkg.build()
    oracle.build()
    binding.lib()


def _vjp(s, eps, abar, pbar, prec, positions="default"):
    o = binding.make_opts(prec, positions=positions)
    n = s.n
    ws = binding.workspace(n, 1, o)
    xb = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    mb = torch.empty(n, dtype=torch.float64, device="cuda")
    binding.nb_forces_vjp(dev(s.pos), dev(s.mass), eps, dev(abar),
                          None if pbar is None else dev(pbar), xb, mb, ws, o)
    assert binding.nb_poll_status(ws, o) == binding.NB_OK
    return host(xb), host(mb)


def _relmax(a, ref):
    return np.abs(a - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("n", [2, 5, 100, 1000, 4099])
@pytest.mark.parametrize("with_pbar", [False, True])
def test_force_vjp_matches_oracle(n, with_pbar):
    s = ics.plummer_lognormal(n, seed=n)
    rng = np.random.default_rng(n)
    abar = rng.normal(size=(n, 3))
    pbar = rng.normal(size=n) if with_pbar else None
    rx, rm = oracle.forces_vjp(s.pos, s.mass, 0.01, abar, pbar)
    # split positions: tight; the default single-float displacement: at the
    # gradient tolerance (1e-4)
    for prec, pos_mode, tol in (("f64acc", "split", 2e-6), ("f64acc", "default", 1e-4),
                                ("fp64", "default", 1e-12)):
        xb, mb = _vjp(s, 0.01, abar, pbar, prec, pos_mode)
        assert _relmax(xb, rx) <= tol and _relmax(mb, rm) <= tol, (prec, pos_mode,
                                                                 _relmax(xb, rx), _relmax(mb, rm))


def test_force_vjp_eps_zero():
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.5, -0.25], [-0.75, 0.25, 0.5], [0.0, 0.0, 0.0]])
    mass = np.array([1.0, 0.5, 0.25, 2.0])
    s = ics.ParticleSet(pos, np.zeros_like(pos), mass)
    abar = np.random.default_rng(1).normal(size=(4, 3))
    pbar = np.random.default_rng(2).normal(size=4)
    rx, rm = oracle.forces_vjp(pos, mass, 0.0, abar, pbar)
    for prec, tol in (("f64acc", 1e-6), ("fp64", 1e-12)):
        xb, mb = _vjp(s, 0.0, abar, pbar, prec)
        assert np.all(np.isfinite(xb)) and np.all(np.isfinite(mb))
        assert _relmax(xb, rx) <= tol and _relmax(mb, rm) <= tol


@pytest.mark.parametrize("mode", ["recompute", "reverse"])
@pytest.mark.parametrize("prec,tol_med,tol_max", [("fp64", 1e-10, 1e-9), ("f64acc", 1e-4, 1e-3)])
def test_trajectory_gradient_matches_oracle(mode, prec, tol_med, tol_max):
    n, eps, h, steps = 256, 0.02, 1e-3, 40
    s = ics.plummer(n, seed=5)
    target = ics.perturb_positions(s.pos, 1e-3, seed=2)
    L, gx, gv, gm = adjoint.loss_and_grads(s.pos, s.vel, s.mass, eps, h, steps, target,
                                           segment=10, precision=prec, mode=mode)
    rL, rx, rv, rm = oracle.trajectory_loss_grad(s.pos, s.vel, s.mass, eps, h, steps, target)
    ours = np.concatenate([host(gx).ravel(), host(gv).ravel(), host(gm)])
    ref = np.concatenate([rx.ravel(), rv.ravel(), rm])
    coords = ics.random_coordinates(n, k=64, seed=3)
    rel = np.abs(ours[coords] - ref[coords]) / np.maximum(np.abs(ref[coords]),
                                                          1e-6 * np.abs(ref).max())
    assert abs(float(L) - rL) <= 1e-9 * abs(rL)
    assert np.median(rel) <= tol_med and rel.max() <= tol_max, (np.median(rel), rel.max())
    assert _relmax(ours, ref) <= tol_max


def test_reverse_and_recompute_agree():
    n, eps, h, steps = 2048, 5e-3, 1e-3, 60
    s = ics.plummer(n, seed=7)
    target = ics.perturb_positions(s.pos, 1e-3, seed=2)
    g = {}
    for mode in ("recompute", "reverse"):
        _, gx, gv, gm = adjoint.loss_and_grads(s.pos, s.vel, s.mass, eps, h, steps, target,
                                               segment=20, mode=mode)
        g[mode] = np.concatenate([host(gx).ravel(), host(gv).ravel(), host(gm)])
    assert _relmax(g["reverse"], g["recompute"]) <= 1e-6
