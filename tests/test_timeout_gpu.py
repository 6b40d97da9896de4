"""Bounded device waits running out, on the GPU, without a fault.

The direct-pair kernels (force, VJP, acceleration + jerk) stage j-tiles
through a ring of shared-memory stages filled by bulk copies that complete
on mbarriers; every wait on a stage is bounded by opts.timeout_cycles.  The
kernels are compute-bound, so in normal operation each stage has landed long
before it is waited on.  The test hook opts.test_unissued_stage = 2 makes
every CTA skip the copies of its second stage: nothing ever completes that
mbarrier phase (a flag that nothing sets), the wait gives up after
timeout_cycles (here ~1 ms), the kernel latches NB_ERR_TIMEOUT, lets the
copies that were issued land, and returns.  The tests check that
nb_poll_status reports the timeout, and that after the caller re-zeroes the
workspace (an interrupted call leaves arrival counters behind, as nbody.h
states) the next call matches the oracle.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2605_02744_gb300 import binding, ics
from tests.gpu_util import TOL, dev, host, rel_err, rel_vec_err

pytestmark = pytest.mark.gpu

SHORT = 2_000_000  # cycles: about 1 ms


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2605_02744_gb300 as pkg
    pkg.build()
    oracle.build()
    binding.lib()


def _timed_out(call, ws, opts):
    """One call with the second ring stage never issued: NB_ERR_TIMEOUT."""
    ws.zero_()
    t0 = time.perf_counter()
    call(binding.make_opts(opts["precision"], positions=opts.get("positions", "default"),
                           pairs="direct", timeout_cycles=SHORT, test_unissued_stage=2))
    rc = binding.nb_poll_status(ws, None)
    took = time.perf_counter() - t0
    assert rc == binding.NB_ERR_TIMEOUT, rc
    assert took < 1.5, took  # the bounded wait, not the 2 s default drain bound
    # the status word was cleared by the poll; re-zero the rest of the workspace
    ws.zero_()
    assert binding.nb_poll_status(ws, None) == binding.NB_OK


@pytest.mark.parametrize("prec", ["kahan", "f64acc"])
def test_force_wait_runs_out_then_recovers(prec):
    n, eps = 20001, 0.01
    s = ics.plummer(n, seed=5)
    pos, mass = dev(s.pos), dev(s.mass)
    acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    o = binding.make_opts(prec, pairs="direct")
    ws = binding.workspace(n, 1, o)

    _timed_out(lambda os_: binding.nb_forces(pos, mass, eps, acc, pot, ws, os_), ws,
               {"precision": prec})
    binding.nb_forces(pos, mass, eps, acc, pot, ws, o)
    assert binding.nb_poll_status(ws, o) == binding.NB_OK
    ra, rp = oracle.forces(s.pos, s.mass, eps)
    assert rel_vec_err(host(acc), ra).max() <= TOL[prec]
    assert rel_err(host(pot), rp).max() <= TOL[prec]


def test_vjp_wait_runs_out_then_recovers():
    n, eps = 9001, 0.02
    s = ics.plummer_lognormal(n, seed=6)
    rng = np.random.default_rng(6)
    abar, pbar = rng.normal(size=(n, 3)), rng.normal(size=n)
    pos, mass, ab, pb = dev(s.pos), dev(s.mass), dev(abar), dev(pbar)
    xb = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    mb = torch.empty(n, dtype=torch.float64, device="cuda")
    o = binding.make_opts("f64acc", positions="split")
    ws = binding.workspace(n, 1, o)

    _timed_out(lambda os_: binding.nb_forces_vjp(pos, mass, eps, ab, pb, xb, mb, ws, os_), ws,
               {"precision": "f64acc", "positions": "split"})
    binding.nb_forces_vjp(pos, mass, eps, ab, pb, xb, mb, ws, o)
    assert binding.nb_poll_status(ws, o) == binding.NB_OK
    rx, rm = oracle.forces_vjp(s.pos, s.mass, eps, abar, pbar)
    assert np.abs(host(xb) - rx).max() / np.abs(rx).max() <= 2e-6
    assert np.abs(host(mb) - rm).max() / np.abs(rm).max() <= 2e-6


def test_jerk_wait_runs_out_then_recovers():
    n, eps = 9001, 0.01
    s = ics.plummer_lognormal(n, seed=7)
    pos, vel, mass = dev(s.pos), dev(s.vel), dev(s.mass)
    acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    jerk = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    o = binding.make_opts("f64acc")
    ws = binding.workspace(n, 1, o)

    _timed_out(lambda os_: binding.nb_forces_jerk(pos, vel, mass, eps, acc, jerk, pot, ws, os_),
               ws, {"precision": "f64acc"})
    binding.nb_forces_jerk(pos, vel, mass, eps, acc, jerk, pot, ws, o)
    assert binding.nb_poll_status(ws, o) == binding.NB_OK
    ra, rj, rp = oracle.forces_jerk(s.pos, s.vel, s.mass, eps)
    assert rel_vec_err(host(acc), ra).max() <= 1e-5
    assert rel_vec_err(host(jerk), rj).max() <= 1e-4
