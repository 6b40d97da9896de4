"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/nbody_oracle.c (a flipped
sign, a dropped softening term, a wrong step factor, a swapped index, a
stale value, a wrong coefficient), builds it, points the oracle at it, and
checks that the named pin test fails.  CPU only.
"""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_adjoint as T_adj
from tests import test_oracle_forces as T_f
from tests import test_oracle_hermite as T_h
from tests import test_oracle_integrator as T_i

SRC = os.path.join(os.path.dirname(oracle.__file__), "nbody_oracle.c")

MUTATIONS = [
    ("potential sign", "        phi -= mass[j] / s;\n    }\n    ai[0]",
     "        phi += mass[j] / s;\n    }\n    ai[0]",
     lambda o: T_f.test_matches_50_digit_brute_force(o, 5, 0.01)),
    ("softening dropped", "dz * dz + eps2;\n        if (s2 == 0.0) continue;\n        const double s = sqrt(s2);\n        const double inv_s3",
     "dz * dz;\n        if (s2 == 0.0) continue;\n        const double s = sqrt(s2);\n        const double inv_s3",
     lambda o: T_f.test_matches_50_digit_brute_force(o, 5, 0.7)),
    ("displacement sign (x)", "const double dx = pos[3 * j] - xi;",
     "const double dx = xi - pos[3 * j];", T_f.test_hand_worked_two_body),
    ("self pair included", "        if (j == i) continue;\n        const double dx",
     "        const double dx", T_f.test_single_particle_and_coincident_pair),
    ("closing kick doubled",
     "        orc_forces(N, pos, mass, eps, G, acc, pot);\n        for (int64_t k = 0; k < 3 * N; ++k) vel[k] += 0.5 * h * acc[k];",
     "        orc_forces(N, pos, mass, eps, G, acc, pot);\n        for (int64_t k = 0; k < 3 * N; ++k) vel[k] += h * acc[k];",
     T_i.test_circular_orbit_one_period_second_order),
    ("stale acceleration in the step",
     "        for (int64_t k = 0; k < 3 * N; ++k) pos[k] += h * vel[k];\n        orc_forces(N, pos, mass, eps, G, acc, pot);",
     "        for (int64_t k = 0; k < 3 * N; ++k) pos[k] += h * vel[k];",
     T_i.test_time_reversibility),
    ("kinetic energy factor", "K += 0.5 * mass[i] * v2;", "K += mass[i] * v2;",
     T_i.test_energy_sums),
    ("VJP mass index", "xb[a] += G * mass[k] * M[3 * b + a] * abar[3 * i + b];",
     "xb[a] += G * mass[i] * M[3 * b + a] * abar[3 * i + b];",
     lambda o: T_adj.test_vjp_matches_autograd(o, False)),
    ("VJP mass-gradient sign", "mb += G * d[a] * is3 * abar[3 * i + a];",
     "mb -= G * d[a] * is3 * abar[3 * i + a];",
     lambda o: T_adj.test_vjp_matches_autograd(o, False)),
    ("jerk coefficient", "jk[c] += mass[j] * (w[c] * inv3 - 3.0 * dw * d[c] * inv3 / s2);\n            }\n            phi",
     "jk[c] += mass[j] * (w[c] * inv3 - 2.0 * dw * d[c] * inv3 / s2);\n            }\n            phi",
     T_h.test_jerk_is_directional_derivative_of_acceleration),
    ("Hermite corrector coefficient", "(acc[k] - a1[k]) * h * h / 12.0;",
     "(acc[k] - a1[k]) * h * h / 10.0;", T_h.test_hermite4_fourth_order_on_kepler_ellipse),
]


@pytest.mark.parametrize("name,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_planted_mistake(tmp_path, oracle_mod, name, old, new, pin):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for '{name}' must occur exactly once"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-std=c11", "-shared",
                    "-fPIC", "-o", str(lib), str(mutant), "-lm"], check=True)
    prev = oracle.use_library(str(lib))
    try:
        with pytest.raises(AssertionError):
            pin(oracle)
    finally:
        oracle.restore_library(prev)
    pin(oracle)  # and the real oracle still passes the same pin
