"""Writes the stored expected values under tests/golden/.

It calls only the oracle package (the 50-digit decimal evaluation, the FP64
leapfrog and its discrete adjoint) and the seeded input generators, never the
CUDA library.  Run from the repository root:

    python tests/golden/make_golden.py            # bruteforce_n6.txt
    python tests/golden/make_golden.py adjoint    # adjoint_c4.txt (minutes)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import hiprec  # noqa: E402


def bruteforce_n6():
    # a fixed, hand-chosen system with dyadic coordinates and masses so the
    # inputs are exact in binary; eps = 0.125, G = 1
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.5, -0.25], [-0.75, 0.25, 0.5],
                    [0.125, -1.0, 0.375], [2.0, 2.0, 2.0], [-0.5, -0.5, 1.5]])
    mass = np.array([1.0, 0.5, 0.25, 2.0, 0.125, 0.75])
    eps = 0.125
    acc, pot = hiprec.forces(pos, mass, eps)
    lines = ["# 50-digit decimal direct sum (Eq. 1, Sec. 2.1; softening r^2 + eps^2),",
             "# rounded to double. eps = 0.125, G = 1.",
             "# columns: x y z m | ax ay az phi"]
    for i in range(6):
        vals = list(pos[i]) + [mass[i]] + list(acc[i]) + [pot[i]]
        lines.append(" ".join(repr(float(v)) for v in vals))
    with open(os.path.join(HERE, "bruteforce_n6.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


def adjoint_c4():
    """The reference gradient of the adjoint workload (16384-particle Plummer
    sphere, eps = 5e-3, 200 KDK steps of 1e-3; target = final positions of an
    FP64 run from positions perturbed by N(0, (1e-3)^2), seed 2): the loss,
    the largest |gradient| over all 7N scalars and the gradient on the 64
    coordinates drawn with seed 3.  A checksum of the target lets the test
    confirm that it rebuilt the same target."""
    import oracle
    from paper_2605_02744_gb300 import ics
    n, eps, h, steps = 16384, 5e-3, 1e-3, 200
    oracle.build()
    s = ics.plummer(n, seed=0)
    xp = ics.perturb_positions(s.pos, 1e-3, seed=2)
    target, _, _, _ = oracle.kdk(xp, s.vel, s.mass, eps, h, steps)
    L, gx, gv, gm = oracle.trajectory_loss_grad(s.pos, s.vel, s.mass, eps, h, steps, target)
    ref = np.concatenate([gx.ravel(), gv.ravel(), gm])
    coords = ics.random_coordinates(n, k=64, seed=3)
    lines = ["# FP64 oracle: KDK leapfrog (Sec. 2.2) and its unmerged discrete adjoint,",
             "# loss = (1/N) sum |x_i(T) - x*_i|^2; N = 16384 Plummer (seed 0), eps = 5e-3,",
             "# h = 1e-3, 200 steps; target from positions perturbed by N(0, (1e-3)^2) (seed 2).",
             "# coordinate c < 3N: x0[c], < 6N: v0[c - 3N], else m[c - 6N]",
             f"target_abs_sum {float(np.abs(target).sum())!r}",
             f"loss {float(L)!r}",
             f"grad_abs_max {float(np.abs(ref).max())!r}"]
    for c in coords:
        lines.append(f"grad {int(c)} {float(ref[c])!r}")
    with open(os.path.join(HERE, "adjoint_c4.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    if sys.argv[1:] == ["adjoint"]:
        adjoint_c4()
    else:
        bruteforce_n6()
