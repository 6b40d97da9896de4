"""The paper's validation check (Sec. 4.1, Fig. 4): the distribution of
per-particle energies at t = 3 from the accelerated run matches the one of
the FP64 reference run, although individual orbits have diverged."""
import numpy as np
import pytest

import oracle
from paper_2605_02744_gb300 import api, binding, diagnostics, ics
from tests.gpu_util import host

pytestmark = pytest.mark.gpu


def test_energy_distribution_at_t3_matches_oracle():
    oracle.build()
    s = ics.plummer(2048, seed=8)
    eps, h, steps = 0.01, 1e-3, 3000
    g = api.System(s.pos, s.vel, s.mass, eps, precision="kahan")
    g.step(h, steps)
    assert g.poll() == binding.NB_OK
    e_gpu = diagnostics.specific_energies(host(g.vel), host(g.pot))
    _, vo, _, po = oracle.kdk(s.pos, s.vel, s.mass, eps, h, steps)
    e_ref = diagnostics.specific_energies(vo, po)
    cmp = diagnostics.compare_distributions(e_gpu, e_ref)
    assert cmp["p"] > 0.05 and cmp["mean_rel"] < 1e-3 and cmp["std_rel"] < 1e-2, cmp
    # the orbits themselves have drifted apart (chaos), the distribution has not
    assert np.abs(host(g.pos)).max() > 0
