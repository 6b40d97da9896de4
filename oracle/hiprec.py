"""50-digit decimal evaluation of the softened direct sum, for N <= 8.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  It pins the FP64 oracle:
the double inputs are converted to Decimal exactly, every operation of
a_i = G sum_{j != i} m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^{3/2} and
phi_i = -G sum_{j != i} m_j / (|x_j - x_i|^2 + eps^2)^{1/2} (Eq. 1, Sec. 2.1,
softening read as r^2 + eps^2) is carried at 50 significant digits, and only
the final values are rounded to double.
"""
from __future__ import annotations

from decimal import Decimal, localcontext

import numpy as np


def forces(pos, mass, eps: float, G: float = 1.0, digits: int = 50):
    pos = np.asarray(pos, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    n = mass.shape[0]
    if n > 8:
        raise ValueError("the 50-digit brute force is meant for N <= 8")
    acc = np.zeros((n, 3))
    pot = np.zeros(n)
    with localcontext() as ctx:
        ctx.prec = digits
        P = [[Decimal(float(pos[i, c])) for c in range(3)] for i in range(n)]
        M = [Decimal(float(m)) for m in mass]
        e2 = Decimal(float(eps)) * Decimal(float(eps))
        g = Decimal(float(G))
        for i in range(n):
            a = [Decimal(0)] * 3
            phi = Decimal(0)
            for j in range(n):
                if j == i:
                    continue
                d = [P[j][c] - P[i][c] for c in range(3)]
                s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + e2
                if s2 == 0:
                    continue
                s = s2.sqrt()
                for c in range(3):
                    a[c] += M[j] * d[c] / (s2 * s)
                phi -= M[j] / s
            for c in range(3):
                acc[i, c] = float(g * a[c])
            pot[i] = float(g * phi)
    return acc, pot
