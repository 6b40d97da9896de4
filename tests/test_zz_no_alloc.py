"""nb_forces_noalloc: the force evaluation for callers that cannot allocate
device memory (and so cannot pass a workspace), checked through the C ABI
against nb_forces on the same inputs, two calls in a row each time.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import pytest
import torch

from paper_2605_02744_gb300 import binding, ics
from tests.gpu_util import TOL, dev, host, rel_err, rel_vec_err


@pytest.fixture(scope="module")
def lib():
    import paper_2605_02744_gb300 as pkg
    pkg.build()
    return binding.lib()


def _call_noalloc(lib, pos, mass, eps, opts):
    n = mass.shape[0]
    acc = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    pot = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.nb_forces_noalloc(pos.data_ptr(), mass.data_ptr(), n, eps, acc.data_ptr(),
                               pot.data_ptr(), ctypes.byref(opts))
    assert rc == binding.NB_OK, binding.nb_last_error()
    return acc, pot


def _call_ws(lib, pos, mass, eps, opts):
    n = mass.shape[0]
    acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = binding.workspace(n, 1, opts)
    rc = lib.nb_forces(pos.data_ptr(), mass.data_ptr(), n, eps, acc.data_ptr(), pot.data_ptr(),
                       ws.data_ptr(), ws.numel(), ctypes.byref(opts))
    assert rc == binding.NB_OK, binding.nb_last_error()
    return acc, pot


def test_rejects_sizes_beyond_its_maximum(lib):
    o = binding.nb_opts()
    lib.nb_opts_default(ctypes.byref(o))
    fake = 1 << 20
    assert lib.nb_forces_noalloc(fake, fake, 32769, 0.01, fake, None, ctypes.byref(o)) == \
        binding.NB_ERR_INVALID
    assert "32768" in binding.nb_last_error()
    assert lib.nb_forces_noalloc(fake, fake, 0, 0.01, fake, None, ctypes.byref(o)) == \
        binding.NB_ERR_INVALID


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["kahan", "f64acc", "fp64"])
@pytest.mark.parametrize("n", [777, 32768])
def test_matches_workspace_entry_point_twice(lib, prec, n):
    opts = binding.make_opts(prec)
    for seed in (1, 2):  # two calls in a row, different inputs
        s = ics.plummer(n, seed=seed)
        pos, mass = dev(s.pos), dev(s.mass)
        a0, p0 = _call_noalloc(lib, pos, mass, 0.01, opts)
        a1, p1 = _call_ws(lib, pos, mass, 0.01, opts)
        torch.cuda.synchronize()
        ea = rel_vec_err(host(a0), host(a1)).max()
        ep = rel_err(host(p0), host(p1)).max()
        assert ea <= TOL[prec] and ep <= TOL[prec], (prec, n, seed, ea, ep)
