"""Bounded device waits running out, on the GPU, without a fault.

The direct-pair kernels (force, VJP, acceleration + jerk) stage j-tiles
through shared memory with bulk copies that complete on mbarriers; every
wait on a stage is bounded by opts.timeout_cycles.  Here the bound is one
clock cycle, so a wait that does not find its stage already complete gives
up: the kernel latches NB_ERR_TIMEOUT in the workspace status word, lets the
copies still in flight land (with at least the default bound), and returns.
The tests check that nb_poll_status reports the timeout, and that after the
caller re-zeroes the workspace (the arrival counters of an interrupted call
are left behind, as nbody.h states) the next call with the default bound
matches the oracle.  Whether a particular wait finds its stage complete
depends on timing (a stage issued long before its wait has landed), so a
call is repeated (with the L2 flushed first) until one reports the timeout.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02744_gb300 import binding, ics
from tests.gpu_util import TOL, dev, host, rel_err, rel_vec_err

pytestmark = pytest.mark.gpu

ATTEMPTS = 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2605_02744_gb300 as pkg
    pkg.build()
    oracle.build()
    binding.lib()


@pytest.fixture(scope="module")
def flush():
    return torch.empty(256 << 20, dtype=torch.uint8, device="cuda")


def _timed_out(call, ws, opts, flush):
    """Runs call(opts_short) until one attempt reports NB_ERR_TIMEOUT."""
    seen = []
    for _ in range(ATTEMPTS):
        ws.zero_()
        flush.zero_()
        call(binding.make_opts(opts["precision"], positions=opts.get("positions", "default"),
                               pairs="direct", timeout_cycles=1))
        rc = binding.nb_poll_status(ws, None)
        seen.append(rc)
        if rc == binding.NB_ERR_TIMEOUT:
            break
    assert binding.NB_ERR_TIMEOUT in seen, seen
    assert all(rc in (binding.NB_OK, binding.NB_ERR_TIMEOUT) for rc in seen), seen
    # the status word was cleared by the poll; re-zero the rest of the workspace
    ws.zero_()
    assert binding.nb_poll_status(ws, None) == binding.NB_OK


@pytest.mark.parametrize("prec", ["kahan", "f64acc"])
def test_force_wait_runs_out_then_recovers(prec, flush):
    n, eps = 20001, 0.01
    s = ics.plummer(n, seed=5)
    pos, mass = dev(s.pos), dev(s.mass)
    acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    o = binding.make_opts(prec, pairs="direct")
    ws = binding.workspace(n, 1, o)

    _timed_out(lambda os_: binding.nb_forces(pos, mass, eps, acc, pot, ws, os_), ws,
               {"precision": prec}, flush)
    binding.nb_forces(pos, mass, eps, acc, pot, ws, o)
    assert binding.nb_poll_status(ws, o) == binding.NB_OK
    ra, rp = oracle.forces(s.pos, s.mass, eps)
    assert rel_vec_err(host(acc), ra).max() <= TOL[prec]
    assert rel_err(host(pot), rp).max() <= TOL[prec]


def test_vjp_wait_runs_out_then_recovers(flush):
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
               {"precision": "f64acc", "positions": "split"}, flush)
    binding.nb_forces_vjp(pos, mass, eps, ab, pb, xb, mb, ws, o)
    assert binding.nb_poll_status(ws, o) == binding.NB_OK
    rx, rm = oracle.forces_vjp(s.pos, s.mass, eps, abar, pbar)
    assert np.abs(host(xb) - rx).max() / np.abs(rx).max() <= 2e-6
    assert np.abs(host(mb) - rm).max() / np.abs(rm).max() <= 2e-6


def test_jerk_wait_runs_out_then_recovers(flush):
    n, eps = 9001, 0.01
    s = ics.plummer_lognormal(n, seed=7)
    pos, vel, mass = dev(s.pos), dev(s.vel), dev(s.mass)
    acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    jerk = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    o = binding.make_opts("f64acc")
    ws = binding.workspace(n, 1, o)

    _timed_out(lambda os_: binding.nb_forces_jerk(pos, vel, mass, eps, acc, jerk, pot, ws, os_),
               ws, {"precision": "f64acc"}, flush)
    binding.nb_forces_jerk(pos, vel, mass, eps, acc, jerk, pot, ws, o)
    assert binding.nb_poll_status(ws, o) == binding.NB_OK
    ra, rj, rp = oracle.forces_jerk(s.pos, s.vel, s.mass, eps)
    assert rel_vec_err(host(acc), ra).max() <= 1e-5
    assert rel_vec_err(host(jerk), rj).max() <= 1e-4
