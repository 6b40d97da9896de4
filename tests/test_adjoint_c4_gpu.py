"""The adjoint workload at full size against the oracle: 16384-particle
Plummer sphere, eps = 5e-3, 200 KDK steps of 1e-3, loss = mean squared
distance of the final positions to a target (the final positions of an FP64
run from positions perturbed by N(0, (1e-3)^2), seed 2), gradients with
respect to the initial positions, velocities and masses through the library
(step checkpoints every 20 steps; time-reversed and recomputed backward
passes), checked on the 64 coordinates drawn with seed 3 from the 7N
scalars:

* FP64-pair gradient vs the oracle's unmerged step adjoint: <= 1e-9;
* FP32-pair, FP64-accumulate gradient vs the oracle: median <= 1e-4,
  max <= 1e-3;
* finite differences of the FP64-pair GPU forward map vs the oracle's
  gradient: <= 1e-6 relative plus the loss's rounding noise over the step
  (central differences with h = 1e-6 for positions and velocities; for
  masses, whose gradients are smallest, a four-point stencil with
  h = 1e-2 m_k, truncation error O(h^4)).

The loss's FP64 rounding noise: the final positions carry ~|x| u sqrt(200)
~ 2e-15 of accumulated rounding, so L = (1/N) sum |x_i - x*_i|^2 with
|x_i - x*_i| ~ 1e-3 moves by ~(2/N) 1e-3 2e-15 sqrt(N) ~ 3e-20 from run to
run of nearly equal inputs; the gate allows ETA = 1e-18 of it per loss
value.  (Step sizes of 1e-6 m_k for masses, first tried, leave that noise
at up to 10 % of their gradients.)  The differences are taken of the GPU's
FP64-pair map, not the oracle's: about 150 oracle runs of 200 steps at this
size take about half an hour on 16 host cores, while the FP64 GPU map
agrees with the oracle's to ~1e-12.

The oracle's reverse pass (200 forward steps and 400 force VJPs, about seven
minutes on 16 host cores) is run once by tests/golden/make_golden.py, which
calls only the oracle and the input generators, and stored in
tests/golden/adjoint_c4.txt; the test rebuilds the target with the oracle and
checks it against the checksum stored beside the gradient.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2605_02744_gb300 import adjoint, api, binding, ics
from tests.gpu_util import host

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N, EPS, H, STEPS, SEGMENT = 16384, 5e-3, 1e-3, 200, 20


def _golden():
    """tests/golden/adjoint_c4.txt, written by tests/golden/make_golden.py from
    the oracle alone: (target checksum, L, max |grad|, {coordinate: grad})."""
    path = os.path.join(os.path.dirname(__file__), "golden", "adjoint_c4.txt")
    vals, grad = {}, {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = line.split()
            if w[0] == "grad":
                grad[int(w[1])] = float(w[2])
            else:
                vals[w[0]] = float(w[1])
    return vals["target_abs_sum"], vals["loss"], vals["grad_abs_max"], grad


@pytest.fixture(scope="module")
def workload():
    import paper_2605_02744_gb300 as pkg
    pkg.build()
    oracle.build()
    binding.lib()
    s = ics.plummer(N, seed=0)
    # the target: an FP64 oracle run from perturbed positions, same v0 and m
    xp = ics.perturb_positions(s.pos, 1e-3, seed=2)
    target, _, _, _ = oracle.kdk(xp, s.vel, s.mass, EPS, H, STEPS)
    tsum, L, gmax, grad = _golden()
    assert abs(np.abs(target).sum() - tsum) <= 1e-12 * tsum
    coords = ics.random_coordinates(N, k=64, seed=3)
    assert sorted(grad) == sorted(int(c) for c in coords)
    ref = np.zeros(7 * N)
    ref[coords] = [grad[int(c)] for c in coords]
    return s, target, L, ref, coords, gmax


def _gpu_grad(s, target, prec, mode):
    L, gx, gv, gm = adjoint.loss_and_grads(s.pos, s.vel, s.mass, EPS, H, STEPS, target,
                                           segment=SEGMENT, precision=prec, mode=mode)
    return float(L), np.concatenate([host(gx).ravel(), host(gv).ravel(), host(gm)])


def _rel(a, ref, gmax):
    # coordinates with a tiny true gradient compare against 1e-6 of the largest
    return np.abs(a - ref) / np.maximum(np.abs(ref), 1e-6 * gmax)


@pytest.mark.parametrize("mode", ["reverse", "recompute"])
def test_fp64_gradient_matches_oracle(workload, mode):
    s, target, rL, ref, coords, gmax = workload
    L, g = _gpu_grad(s, target, "fp64", mode)
    assert abs(L - rL) <= 1e-9 * abs(rL), (L, rL)
    rel = _rel(g[coords], ref[coords], gmax)
    assert rel.max() <= 1e-9, (mode, rel.max())


@pytest.mark.parametrize("mode", ["reverse", "recompute"])
def test_f64acc_gradient_matches_oracle(workload, mode):
    s, target, rL, ref, coords, gmax = workload
    _, g = _gpu_grad(s, target, "f64acc", mode)
    rel = _rel(g[coords], ref[coords], gmax)
    assert np.median(rel) <= 1e-4 and rel.max() <= 1e-3, (mode, np.median(rel), rel.max())


ETA = 1e-18  # bound on the FP64 rounding noise of one loss value


def test_finite_differences_match_oracle_gradient(workload):
    s, target, _, ref, coords, _ = workload
    sysm = api.System(s.pos, s.vel, s.mass, EPS, precision="fp64", pairs="symmetric")
    tgt = torch.tensor(target, device="cuda")

    def loss(p, v, m):
        sysm.pos.copy_(torch.tensor(p, device="cuda"))
        sysm.vel.copy_(torch.tensor(v, device="cuda"))
        sysm.mass.copy_(torch.tensor(m, device="cuda"))
        sysm.state.acc_valid = 0
        sysm.step(H, STEPS)
        return float(((sysm.pos - tgt) ** 2).sum() / N)

    def shifted(c, d):
        p, v, m = s.pos.copy(), s.vel.copy(), s.mass.copy()
        if c < 3 * N:
            p.reshape(-1)[c] += d
        elif c < 6 * N:
            v.reshape(-1)[c - 3 * N] += d
        else:
            m[c - 6 * N] += d
        return loss(p, v, m)

    bad = []
    for c in coords:
        g = ref[c]
        if c < 6 * N:
            h = 1e-6
            fd = (shifted(c, h) - shifted(c, -h)) / (2 * h)
            noise = ETA / h
        else:
            h = 1e-2 * s.mass[c - 6 * N]
            fd = (8 * (shifted(c, h) - shifted(c, -h)) - (shifted(c, 2 * h) - shifted(c, -2 * h))) \
                / (12 * h)
            noise = 1.5 * ETA / h
        if abs(fd - g) > 1e-6 * abs(g) + noise:
            bad.append((int(c), fd, g, noise))
    assert binding.NB_OK == sysm.poll()
    assert not bad, bad
