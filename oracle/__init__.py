"""FP64 CPU oracle for the direct N-body hot path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the benchmark's timed CPU-baseline leg may import this package.  The
product library never calls it, and it imports nothing from the product
package: the two share only the seeded input generators.

Contents
--------
* ``nbody_oracle.c`` -- plain double-precision C (OpenMP over the output index
  only): forces + potential (Eq. 1 of Sec. 2.1 with Plummer softening), exact
  rows for a subset, kick-drift-kick leapfrog, energy, the force
  vector-Jacobian product written block by block from the chain rule, and
  acceleration + jerk (App. A, Algorithm 3) with a fourth-order Hermite
  predictor-corrector.
* this module -- ctypes wrappers, the discrete adjoint of one KDK step taken
  term by term (two separate force VJPs per step, never merged), the adjoint
  of a whole trajectory, and the final-position loss.
* ``hiprec`` -- the same force definition in 50-digit decimal arithmetic for
  N <= 8, used to pin the FP64 code.

Pins (all in ``tests/test_oracle_*.py``, run with ``-m "not gpu"``): the
50-digit brute force; the zero-total-force invariant sum_i m_i a_i = 0;
translation, permutation and scaling laws; the two-body closed form; the
Kepler orbit (circular and e = 0.5) for the integrator with its h^2
convergence, angular-momentum conservation and time reversibility; Plummer
statistics for the generator; torch float64 autograd, central finite
differences and the dot-product test for the adjoint.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbody_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile nbody_oracle.c into oracle/_build/liboracle.so with gcc.

    -ffp-contract=off keeps a*b+c unfused on every host, so x86_64 and aarch64
    builds give identical results.
    """
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    """Declares the C signatures on a loaded oracle library."""
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_set_num_threads.argtypes = [ctypes.c_int]
    lib.orc_forces.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp,
                               _dp]
    lib.orc_forces_rows.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int64, _i64p, _dp, _dp]
    lib.orc_kdk.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, ctypes.c_int64, ctypes.c_int, _dp, _dp]
    lib.orc_energy.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp]
    lib.orc_forces_vjp.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                   _dp, _dp, _dp, _dp]
    lib.orc_forces_jerk.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double,
                                    ctypes.c_double, _dp, _dp, _dp]
    lib.orc_forces_jerk_rows.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int64, _i64p, _dp, _dp]
    lib.orc_hermite4.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                                 _dp, _dp]
    return lib


def use_library(path):
    """Swaps the oracle to another build of nbody_oracle.c (the mutation
    tests plant mistakes in a copy to show the pins catch them); returns the
    previous library so the caller can restore it with ``restore_library``."""
    global _lib
    with _lock:
        prev = _lib
        _lib = _configure(ctypes.CDLL(path))
    return prev


def restore_library(prev):
    global _lib
    with _lock:
        _lib = prev


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            _configure(lib)
            _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def forces(pos, mass, eps: float, G: float = 1.0):
    """(acc [N,3], pot [N]) from the softened direct sum (Eq. 1, Sec. 2.1)."""
    mass = _f64(mass)
    n = mass.shape[0]
    pos = _f64(pos, (n, 3))
    acc = np.empty((n, 3))
    pot = np.empty(n)
    _load().orc_forces(n, _ptr(pos), _ptr(mass), float(eps), float(G), _ptr(acc), _ptr(pot))
    return acc, pot


def forces_rows(pos, mass, eps: float, rows, G: float = 1.0):
    """Exact (acc, pot) for the particles listed in ``rows`` against all N."""
    mass = _f64(mass)
    n = mass.shape[0]
    pos = _f64(pos, (n, 3))
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= n):
        raise ValueError("row index out of range")
    acc = np.empty((rows.size, 3))
    pot = np.empty(rows.size)
    _load().orc_forces_rows(n, _ptr(pos), _ptr(mass), float(eps), float(G), rows.size,
                            rows.ctypes.data_as(_i64p), _ptr(acc), _ptr(pot))
    return acc, pot


def kdk(pos, vel, mass, eps: float, h: float, nsteps: int, G: float = 1.0, acc=None):
    """nsteps kick-drift-kick steps; returns (pos, vel, acc, pot) at the end."""
    mass = _f64(mass)
    n = mass.shape[0]
    pos = _f64(pos, (n, 3)).copy()
    vel = _f64(vel, (n, 3)).copy()
    valid = acc is not None
    acc = _f64(acc, (n, 3)).copy() if valid else np.empty((n, 3))
    pot = np.empty(n)
    _load().orc_kdk(n, _ptr(pos), _ptr(vel), _ptr(mass), float(eps), float(G), float(h),
                    int(nsteps), int(valid), _ptr(acc), _ptr(pot))
    if nsteps == 0 and valid:
        _, pot = forces(pos, mass, eps, G)
    return pos, vel, acc, pot


def energy(vel, mass, pot):
    """(K, W, E) with K = 1/2 sum m v^2, W = 1/2 sum m phi."""
    mass = _f64(mass)
    n = mass.shape[0]
    vel = _f64(vel, (n, 3))
    pot = _f64(pot, (n,))
    out = np.empty(3)
    _load().orc_energy(n, _ptr(vel), _ptr(mass), _ptr(pot), _ptr(out))
    return float(out[0]), float(out[1]), float(out[2])


def forces_vjp(pos, mass, eps: float, abar, phibar=None, G: float = 1.0):
    """(xbar [N,3], mbar [N]) = VJP of (a, phi) w.r.t. (x, m) at (pos, mass)."""
    mass = _f64(mass)
    n = mass.shape[0]
    pos = _f64(pos, (n, 3))
    abar = _f64(abar, (n, 3))
    phibar = None if phibar is None else _f64(phibar, (n,))
    xbar = np.empty((n, 3))
    mbar = np.empty(n)
    _load().orc_forces_vjp(n, _ptr(pos), _ptr(mass), float(eps), float(G), _ptr(abar),
                           _ptr(phibar), _ptr(xbar), _ptr(mbar))
    return xbar, mbar


def forces_jerk(pos, vel, mass, eps: float, G: float = 1.0):
    """(acc, jerk, pot): the quantities of App. A, Algorithm 3 (+ potential)."""
    mass = _f64(mass)
    n = mass.shape[0]
    pos = _f64(pos, (n, 3))
    vel = _f64(vel, (n, 3))
    acc = np.empty((n, 3))
    jerk = np.empty((n, 3))
    pot = np.empty(n)
    _load().orc_forces_jerk(n, _ptr(pos), _ptr(vel), _ptr(mass), float(eps), float(G),
                            _ptr(acc), _ptr(jerk), _ptr(pot))
    return acc, jerk, pot


def forces_jerk_rows(pos, vel, mass, eps: float, rows, G: float = 1.0):
    """Exact (acc, jerk) for the particles listed in ``rows`` against all N."""
    mass = _f64(mass)
    n = mass.shape[0]
    pos = _f64(pos, (n, 3))
    vel = _f64(vel, (n, 3))
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    acc = np.empty((rows.size, 3))
    jerk = np.empty((rows.size, 3))
    _load().orc_forces_jerk_rows(n, _ptr(pos), _ptr(vel), _ptr(mass), float(eps), float(G),
                                 rows.size, rows.ctypes.data_as(_i64p), _ptr(acc), _ptr(jerk))
    return acc, jerk


def hermite4(pos, vel, mass, eps: float, h: float, nsteps: int, G: float = 1.0):
    """nsteps of fourth-order Hermite; returns (pos, vel, acc, jerk)."""
    mass = _f64(mass)
    n = mass.shape[0]
    pos = _f64(pos, (n, 3)).copy()
    vel = _f64(vel, (n, 3)).copy()
    acc = np.empty((n, 3))
    jerk = np.empty((n, 3))
    _load().orc_hermite4(n, _ptr(pos), _ptr(vel), _ptr(mass), float(eps), float(G), float(h),
                         int(nsteps), 0, _ptr(acc), _ptr(jerk))
    return pos, vel, acc, jerk


def kdk_step_adjoint(x_n, x_np1, mass, eps: float, h: float, xbar, vbar, mbar, G: float = 1.0):
    """Discrete adjoint of one KDK step, unmerged.

    Forward:  v' = v + (h/2) a(x, m);  x1 = x + h v';  v1 = v' + (h/2) a(x1, m).
    Reverse, given (xbar, vbar) = cotangents of (x1, v1), accumulating mbar:
      1. vbar' = vbar;  u = (h/2) vbar;  xbar += J_x(x1)^T u;  mbar += J_m(x1)^T u
      2. vbar' += h xbar            (the drift);  xbar now belongs to x
      3. w = (h/2) vbar';  xbar += J_x(x)^T w;  mbar += J_m(x)^T w
      4. vbar = vbar'
    Returns the cotangents of (x, v) and the updated mbar.
    """
    u = 0.5 * h * vbar
    gx, gm = forces_vjp(x_np1, mass, eps, u, None, G)
    xbar = xbar + gx
    mbar = mbar + gm
    vhalf = vbar + h * xbar
    w = 0.5 * h * vhalf
    gx, gm = forces_vjp(x_n, mass, eps, w, None, G)
    return xbar + gx, vhalf.copy(), mbar + gm


def trajectory(pos, vel, mass, eps: float, h: float, nsteps: int, G: float = 1.0):
    """Positions x_0 .. x_nsteps ([nsteps+1, N, 3]) and the final velocity."""
    xs = [np.array(pos, dtype=np.float64)]
    x, v, a = np.array(pos, dtype=np.float64), np.array(vel, dtype=np.float64), None
    for _ in range(nsteps):
        x, v, a, _ = kdk(x, v, mass, eps, h, 1, G, acc=a)
        xs.append(x)
    return np.stack(xs), v


def loss_final_positions(x_final, target) -> float:
    """L = (1/N) sum_i |x_i(T) - x*_i|^2."""
    d = np.asarray(x_final) - np.asarray(target)
    return float((d * d).sum() / d.shape[0])


def trajectory_loss_grad(pos, vel, mass, eps: float, h: float, nsteps: int, target,
                         G: float = 1.0):
    """(L, dL/dx0, dL/dv0, dL/dm) through nsteps KDK steps, step adjoints unmerged."""
    xs, _ = trajectory(pos, vel, mass, eps, h, nsteps, G)
    n = xs.shape[1]
    L = loss_final_positions(xs[-1], target)
    xbar = 2.0 / n * (xs[-1] - np.asarray(target))
    vbar = np.zeros_like(xbar)
    mbar = np.zeros(n)
    for k in range(nsteps - 1, -1, -1):
        xbar, vbar, mbar = kdk_step_adjoint(xs[k], xs[k + 1], mass, eps, h, xbar, vbar,
                                            mbar, G)
    return L, xbar, vbar, mbar


def final_loss(pos, vel, mass, eps: float, h: float, nsteps: int, target, G: float = 1.0):
    """The loss alone (used for finite differences)."""
    x, _, _, _ = kdk(pos, vel, mass, eps, h, nsteps, G)
    return loss_final_positions(x, target)
