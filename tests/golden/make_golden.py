"""Writes the stored expected values under tests/golden/.

It calls only the oracle package (the 50-digit decimal evaluation), never the
CUDA library.  Run from the repository root:  python tests/golden/make_golden.py
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


if __name__ == "__main__":
    bruteforce_n6()
