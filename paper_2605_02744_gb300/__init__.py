"""GB300 (sm_103a) direct-summation N-body hot path.

All-pairs softened gravitational acceleration and potential (Eq. 1, Sec. 2.1)
in hand-written CUDA kernels behind a C ABI (include/nbody.h), driven by
kick-drift-kick leapfrog, with its discrete adjoint.  This package holds:

* ``binding``  -- ctypes binding with the C names (nb_forces, nb_step, ...);
* ``api``      -- tensor-level conveniences that allocate outputs/workspace
                  with torch and call the binding;
* ``adjoint``  -- torch.autograd.Function over the step adjoint with
                  segment checkpointing;
* ``tune``     -- the launch-shape autotuner and its JSON cache;
* ``ics``      -- seeded synthetic initial conditions (Plummer spheres).

Submodules load lazily so that ``ics`` can be used without the library.
"""
import importlib

__all__ = ["binding", "api", "adjoint", "tune", "ics", "build"]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libnbody.so in-tree (nvcc, sm_103a)."""
    from . import _build
    return _build.build(force=force, verbose=verbose)


def __getattr__(name):
    if name in ("binding", "api", "adjoint", "tune", "ics"):
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
