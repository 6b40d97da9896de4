"""nb_forces_noalloc: the force evaluation for callers that cannot allocate
device memory (and so cannot pass a workspace), checked through the C ABI
against the FP64 oracle and against nb_forces on the same inputs, two calls
in a row each time.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2605_02744_gb300 import binding, ics
from tests.gpu_util import TOL, dev, host, rel_err, rel_vec_err

GUARD_ROWS = 64
SENTINEL = 12345.678


@pytest.fixture(scope="module")
def lib():
    import paper_2605_02744_gb300 as pkg
    pkg.build()
    return binding.lib()


def _call_noalloc(lib, pos, mass, eps, opts):
    """Outputs with a guard tail: rows past N must come back untouched."""
    n = mass.shape[0]
    acc = torch.full((n + GUARD_ROWS, 3), SENTINEL, dtype=torch.float64, device="cuda")
    pot = torch.full((n + GUARD_ROWS,), SENTINEL, dtype=torch.float64, device="cuda")
    rc = lib.nb_forces_noalloc(pos.data_ptr(), mass.data_ptr(), n, eps, acc.data_ptr(),
                               pot.data_ptr(), ctypes.byref(opts))
    assert rc == binding.NB_OK, binding.nb_last_error()
    assert binding.nb_poll_status(None, opts) == binding.NB_OK, binding.nb_last_error()
    a, p = host(acc), host(pot)
    assert np.all(a[n:] == SENTINEL) and np.all(p[n:] == SENTINEL), "wrote past N"
    return a[:n], p[:n]


def _call_ws(lib, pos, mass, eps, opts):
    n = mass.shape[0]
    acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = binding.workspace(n, 1, opts)
    rc = lib.nb_forces(pos.data_ptr(), mass.data_ptr(), n, eps, acc.data_ptr(), pot.data_ptr(),
                       ws.data_ptr(), ws.numel(), ctypes.byref(opts))
    assert rc == binding.NB_OK, binding.nb_last_error()
    torch.cuda.synchronize()
    return host(acc), host(pot)


def _opts(**kw):
    o = binding.nb_opts()
    binding.lib().nb_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def test_rejects_sizes_beyond_its_maximum(lib):
    o = _opts()
    fake = 1 << 20
    assert lib.nb_forces_noalloc(fake, fake, 32769, 0.01, fake, None, ctypes.byref(o)) == \
        binding.NB_ERR_INVALID
    assert "32768" in binding.nb_last_error()
    assert lib.nb_forces_noalloc(fake, fake, 0, 0.01, fake, None, ctypes.byref(o)) == \
        binding.NB_ERR_INVALID


def test_refuses_options_it_does_not_serve(lib):
    # checked on the host before the fixed array is touched: no GPU needed
    fake = 1 << 20
    tune = binding.nb_tune(threads=128)
    for o in (_opts(pairs=binding.NB_PAIRS_SYMMETRIC),
              _opts(positions=binding.NB_POS_ADAPTIVE),
              _opts(tune=ctypes.pointer(tune))):
        rc = lib.nb_forces_noalloc(fake, fake, 100, 0.01, fake, None, ctypes.byref(o))
        assert rc == binding.NB_ERR_UNSUPPORTED, binding.nb_last_error()


_CASES = [("kahan", "default", 0.01), ("f64acc", "default", 0.01), ("fp64", "default", 0.01),
          ("fp32", "split", 0.01), ("kahan", "default", 0.0)]


@pytest.mark.gpu
@pytest.mark.parametrize("prec,positions,eps", _CASES)
@pytest.mark.parametrize("n", [777, 32768])
def test_matches_oracle_and_workspace_entry_point_twice(lib, oracle_mod, prec, positions, eps, n):
    if eps == 0.0 and n > 777:
        pytest.skip("the unsoftened case runs at the small size only")
    opts = binding.make_opts(prec, positions=positions)
    for seed in (1, 2):  # two calls in a row, different inputs
        s = ics.plummer(n, seed=seed)
        pos, mass = dev(s.pos), dev(s.mass)
        a0, p0 = _call_noalloc(lib, pos, mass, eps, opts)
        ra, rp = oracle_mod.forces(s.pos, s.mass, eps)
        ea = rel_vec_err(a0, ra).max()
        ep = rel_err(p0, rp).max()
        assert ea <= TOL[prec] and ep <= TOL[prec], ("oracle", prec, n, seed, ea, ep)
        a1, p1 = _call_ws(lib, pos, mass, eps, opts)
        ea = rel_vec_err(a0, a1).max()
        ep = rel_err(p0, p1).max()
        assert ea <= TOL[prec] and ep <= TOL[prec], ("nb_forces", prec, n, seed, ea, ep)
