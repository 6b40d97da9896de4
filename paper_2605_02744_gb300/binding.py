"""ctypes binding of libnbody.so (include/nbody.h), same names as the C ABI.

Argument marshalling only: torch CUDA tensors are passed as device pointers
(``data_ptr()``), torch streams as ``cudaStream_t`` handles, and every step
of the computation runs in the library's CUDA kernels.  There is no CPU
fallback: if the library is missing the import of this module succeeds but
the first call raises ``NbLibraryMissing``.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libnbody.so")

NB_OK = 0
NB_ERR_INVALID = 1
NB_ERR_CUDA = 2
NB_ERR_WORKSPACE = 3
NB_ERR_UNSUPPORTED = 4
NB_ERR_TIMEOUT = 5
NB_ERR_NONFINITE = 6

NB_PREC_FP32 = 0
NB_PREC_KAHAN = 1
NB_PREC_F64ACC = 2
NB_PREC_FP64 = 3
PRECISIONS = {"fp32": NB_PREC_FP32, "kahan": NB_PREC_KAHAN, "f64acc": NB_PREC_F64ACC,
              "fp64": NB_PREC_FP64}
NB_POS_DEFAULT = 0
NB_POS_SPLIT = 1
NB_POS_SINGLE = 2
NB_POS_ADAPTIVE = 3
POSITIONS = {"default": NB_POS_DEFAULT, "split": NB_POS_SPLIT, "single": NB_POS_SINGLE,
             "adaptive": NB_POS_ADAPTIVE}
NB_PAIRS_DEFAULT = 0
NB_PAIRS_DIRECT = 1
NB_PAIRS_SYMMETRIC = 2
PAIRS = {"default": NB_PAIRS_DEFAULT, "direct": NB_PAIRS_DIRECT,
         "symmetric": NB_PAIRS_SYMMETRIC}

EXPORTED = ("nb_opts_default", "nb_version", "nb_last_error", "nb_tune_valid",
            "nb_workspace_bytes", "nb_forces", "nb_forces_batched", "nb_step", "nb_energy",
            "nb_forces_vjp", "nb_step_vjp", "nb_step_vjp_reverse", "nb_poll_status",
            "nb_forces_noalloc", "nb_launch_count", "nb_forces_jerk", "nb_hermite4",
            "nb_kernel_timing", "nb_kernel_time", "nb_forces_range", "nb_kick_drift",
            "nb_check_fp_conversions", "nb_forces_vjp_range")


class NbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class NbLibraryMissing(RuntimeError):
    pass


class nb_tune(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("i_per_thread", ctypes.c_int32),
                ("tile_j", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("cluster_ctas", ctypes.c_int32),
                ("item_blocks", ctypes.c_int32)]


class nb_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("G", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("use_graph", ctypes.c_int32),
                ("tune", ctypes.POINTER(nb_tune)), ("timeout_cycles", ctypes.c_int64),
                ("positions", ctypes.c_int32), ("near_gamma", ctypes.c_float),
                ("pairs", ctypes.c_int32), ("test_unissued_stage", ctypes.c_int32)]


class nb_state(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("B", ctypes.c_int32), ("offsets", ctypes.c_void_p),
                ("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("mass", ctypes.c_void_p),
                ("acc", ctypes.c_void_p), ("pot", ctypes.c_void_p), ("eps_b", ctypes.c_void_p),
                ("eps", ctypes.c_double), ("step", ctypes.c_int64),
                ("acc_valid", ctypes.c_int32), ("ws", ctypes.c_void_p),
                ("ws_bytes", ctypes.c_size_t)]


_lib = None
_lock = threading.Lock()
_vp, _d, _i64, _i32, _sz = (ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int32,
                            ctypes.c_size_t)
_OPTS = ctypes.POINTER(nb_opts)
_STATE = ctypes.POINTER(nb_state)

_SIGS = {
    "nb_opts_default": (None, [_OPTS]),
    "nb_version": (ctypes.c_char_p, []),
    "nb_last_error": (ctypes.c_char_p, []),
    "nb_check_fp_conversions": (ctypes.c_int, [_i64, ctypes.c_uint64, ctypes.POINTER(_i64)]),
    "nb_launch_count": (ctypes.c_ulonglong, []),
    "nb_kernel_timing": (ctypes.c_int, [_i32]),
    "nb_kernel_time": (ctypes.c_int, [ctypes.POINTER(_d), ctypes.POINTER(_i64)]),
    "nb_tune_valid": (ctypes.c_int, [ctypes.POINTER(nb_tune)]),
    "nb_workspace_bytes": (_sz, [_i64, _i32, _OPTS]),
    "nb_forces": (ctypes.c_int, [_vp, _vp, _i64, _d, _vp, _vp, _vp, _sz, _OPTS]),
    "nb_forces_batched": (ctypes.c_int, [_vp, _vp, _vp, _i32, _i64, _vp, _vp, _vp, _vp, _sz,
                                         _OPTS]),
    "nb_step": (ctypes.c_int, [_STATE, _d, _i64, _OPTS]),
    "nb_energy": (ctypes.c_int, [_STATE, _vp, _OPTS]),
    "nb_forces_vjp": (ctypes.c_int, [_vp, _vp, _i64, _d, _vp, _vp, _vp, _vp, _vp, _sz, _OPTS]),
    "nb_forces_vjp_range": (ctypes.c_int, [_vp, _vp, _i64, _i64, _i64, _d, _d, _vp, _vp, _vp,
                                           _vp, _vp, _sz, _OPTS]),
    "nb_step_vjp": (ctypes.c_int, [_vp, _vp, _i64, _d, _d, _d, _vp, _vp, _vp, _vp, _sz, _OPTS]),
    "nb_step_vjp_reverse": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _d, _d, _d, _d, _d, _vp, _vp,
                                           _vp, _vp, _sz, _OPTS]),
    "nb_poll_status": (ctypes.c_int, [_vp, _sz, _vp]),
    "nb_forces_noalloc": (ctypes.c_int, [_vp, _vp, _i64, _d, _vp, _vp, _OPTS]),
    "nb_forces_jerk": (ctypes.c_int, [_vp, _vp, _vp, _i64, _d, _vp, _vp, _vp, _vp, _sz, _OPTS]),
    "nb_hermite4": (ctypes.c_int, [_vp, _vp, _vp, _i64, _d, _vp, _vp, _i32, _d, _i64, _vp, _sz,
                                   _OPTS]),
    "nb_forces_range": (ctypes.c_int, [_vp, _vp, _i64, _i64, _i64, _d, _vp, _vp, _vp, _sz,
                                       _OPTS]),
    "nb_kick_drift": (ctypes.c_int, [_vp, _vp, _vp, _i64, _d, _d, _OPTS]),
}


def lib():
    """The loaded library; raises NbLibraryMissing if it was never built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise NbLibraryMissing(
                    f"{LIB_PATH} is missing: build it with paper_2605_02744_gb300.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc != NB_OK:
        raise NbError(rc, lib().nb_last_error().decode())


def _dptr(t, name, dtype=None, optional=False):
    """Device pointer of a contiguous CUDA tensor (or None when optional)."""
    if t is None:
        if optional:
            return None
        raise TypeError(f"{name} is required")
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def make_opts(precision="f64acc", G: float = 1.0, stream=None, use_graph: bool = False,
              tune=None, timeout_cycles: int = 0, positions="default",
              near_gamma: float = 0.0, pairs="default", test_unissued_stage: int = 0) -> nb_opts:
    """nb_opts for a call; stream None = torch's current stream on the current device."""
    o = nb_opts()
    lib().nb_opts_default(ctypes.byref(o))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.G = float(G)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    o.stream = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    o.use_graph = int(bool(use_graph))
    if tune is not None:
        if not isinstance(tune, nb_tune):
            tune = nb_tune(**tune)
        o._tune_ref = tune  # keep alive
        o.tune = ctypes.pointer(tune)
    o.timeout_cycles = int(timeout_cycles)
    o.positions = POSITIONS[positions] if isinstance(positions, str) else int(positions)
    o.near_gamma = float(near_gamma)
    o.pairs = PAIRS[pairs] if isinstance(pairs, str) else int(pairs)
    o.test_unissued_stage = int(test_unissued_stage)
    return o


def nb_version() -> str:
    return lib().nb_version().decode()


def nb_last_error() -> str:
    return lib().nb_last_error().decode()


def nb_check_fp_conversions(n: int, seed: int = 0) -> int:
    """Mismatches of the integer-pipe float <-> double conversions and
    finiteness test against the C ones (edge cases and seeded patterns)."""
    out = _i64(0)
    _check(lib().nb_check_fp_conversions(int(n), int(seed), ctypes.byref(out)))
    return int(out.value)


def nb_launch_count() -> int:
    return int(lib().nb_launch_count())


def nb_kernel_timing(enable: bool) -> None:
    _check(lib().nb_kernel_timing(1 if enable else 0))


def nb_kernel_time():
    """(summed ms, launches) of the pair-kernel launches timed since
    nb_kernel_timing(True)."""
    ms = _d(0.0)
    n = _i64(0)
    _check(lib().nb_kernel_time(ctypes.byref(ms), ctypes.byref(n)))
    return float(ms.value), int(n.value)


def nb_tune_valid(tune) -> bool:
    if not isinstance(tune, nb_tune):
        tune = nb_tune(**tune)
    return bool(lib().nb_tune_valid(ctypes.byref(tune)))


def nb_workspace_bytes(N: int, B: int = 1, opts: nb_opts | None = None) -> int:
    return int(lib().nb_workspace_bytes(int(N), int(B), ctypes.byref(opts) if opts else None))


def workspace(N: int, B: int = 1, opts: nb_opts | None = None, device=None):
    """A zero-filled uint8 CUDA tensor of nb_workspace_bytes(N, B) bytes."""
    import torch
    nbytes = nb_workspace_bytes(N, B, opts)
    return torch.zeros(nbytes, dtype=torch.uint8, device=device or "cuda")


def nb_forces(pos, mass, eps: float, acc, pot, ws, opts: nb_opts):
    import torch
    f64 = torch.float64
    n = mass.shape[0]
    _check(lib().nb_forces(_dptr(pos, "pos", f64), _dptr(mass, "mass", f64), n, float(eps),
                           _dptr(acc, "acc", f64), _dptr(pot, "pot", f64, True),
                           _dptr(ws, "ws"), ws.numel() * ws.element_size(), ctypes.byref(opts)))


def nb_forces_range(pos, mass, i0: int, i1: int, eps: float, acc, pot, ws, opts: nb_opts):
    """Rows i0..i1-1 of the forces of all N particles (acc/pot hold i1-i0 rows)."""
    import torch
    f64 = torch.float64
    n = mass.shape[0]
    _check(lib().nb_forces_range(_dptr(pos, "pos", f64), _dptr(mass, "mass", f64), n, int(i0),
                                 int(i1), float(eps), _dptr(acc, "acc", f64),
                                 _dptr(pot, "pot", f64, True), _dptr(ws, "ws"),
                                 ws.numel() * ws.element_size(), ctypes.byref(opts)))


def nb_kick_drift(pos, vel, acc, kick: float, drift: float, opts: nb_opts):
    """vel += kick acc; pos += drift vel (n = rows of vel)."""
    import torch
    f64 = torch.float64
    _check(lib().nb_kick_drift(_dptr(pos, "pos", f64), _dptr(vel, "vel", f64),
                               _dptr(acc, "acc", f64), vel.shape[0], float(kick), float(drift),
                               ctypes.byref(opts)))


def nb_forces_noalloc(pos, mass, eps: float, acc, pot, opts: nb_opts):
    """nb_forces without a workspace, for callers that may not allocate
    device memory (N <= 32768; scratch is a fixed array in the library)."""
    import torch
    f64 = torch.float64
    n = mass.shape[0]
    _check(lib().nb_forces_noalloc(_dptr(pos, "pos", f64), _dptr(mass, "mass", f64), n,
                                   float(eps), _dptr(acc, "acc", f64),
                                   _dptr(pot, "pot", f64, True), ctypes.byref(opts)))


def nb_forces_batched(pos, mass, offsets, eps, acc, pot, ws, opts: nb_opts):
    import torch
    f64 = torch.float64
    B = offsets.shape[0] - 1
    _check(lib().nb_forces_batched(
        _dptr(pos, "pos", f64), _dptr(mass, "mass", f64), _dptr(offsets, "offsets", torch.int64),
        B, mass.shape[0], _dptr(eps, "eps", f64), _dptr(acc, "acc", f64), _dptr(pot, "pot", f64, True),
        _dptr(ws, "ws"), ws.numel() * ws.element_size(), ctypes.byref(opts)))


def nb_step(state: nb_state, dt: float, nsteps: int, opts: nb_opts):
    _check(lib().nb_step(ctypes.byref(state), float(dt), int(nsteps), ctypes.byref(opts)))


def nb_energy(state: nb_state, out3, opts: nb_opts):
    import torch
    _check(lib().nb_energy(ctypes.byref(state), _dptr(out3, "out3", torch.float64),
                           ctypes.byref(opts)))


def nb_forces_vjp(pos, mass, eps: float, acc_bar, pot_bar, pos_bar, mass_bar, ws, opts: nb_opts):
    import torch
    f64 = torch.float64
    n = mass.shape[0]
    _check(lib().nb_forces_vjp(
        _dptr(pos, "pos", f64), _dptr(mass, "mass", f64), n, float(eps),
        _dptr(acc_bar, "acc_bar", f64), _dptr(pot_bar, "pot_bar", f64, True),
        _dptr(pos_bar, "pos_bar", f64), _dptr(mass_bar, "mass_bar", f64), _dptr(ws, "ws"),
        ws.numel() * ws.element_size(), ctypes.byref(opts)))


def nb_forces_vjp_range(pos, mass, i0: int, i1: int, eps: float, coef: float, acc_bar, pot_bar,
                        pos_bar, mass_bar, ws, opts: nb_opts):
    """pos_bar / mass_bar (i1-i0 rows) += coef x the VJP rows i0..i1-1 of
    the cotangents acc_bar / pot_bar of all N particles."""
    import torch
    f64 = torch.float64
    n = mass.shape[0]
    _check(lib().nb_forces_vjp_range(
        _dptr(pos, "pos", f64), _dptr(mass, "mass", f64), n, int(i0), int(i1), float(eps),
        float(coef), _dptr(acc_bar, "acc_bar", f64), _dptr(pot_bar, "pot_bar", f64, True),
        _dptr(pos_bar, "pos_bar", f64), _dptr(mass_bar, "mass_bar", f64), _dptr(ws, "ws"),
        ws.numel() * ws.element_size(), ctypes.byref(opts)))


def nb_step_vjp(pos_k, mass, eps: float, drift_dt: float, kick_coef: float, pos_bar, vel_bar,
                mass_bar, ws, opts: nb_opts):
    import torch
    f64 = torch.float64
    n = mass.shape[0]
    _check(lib().nb_step_vjp(
        _dptr(pos_k, "pos_k", f64), _dptr(mass, "mass", f64), n, float(eps), float(drift_dt),
        float(kick_coef), _dptr(pos_bar, "pos_bar", f64), _dptr(vel_bar, "vel_bar", f64),
        _dptr(mass_bar, "mass_bar", f64), _dptr(ws, "ws"), ws.numel() * ws.element_size(),
        ctypes.byref(opts)))


def nb_step_vjp_reverse(pos, vhalf, acc, mass, eps: float, rewind_kick: float,
                        rewind_drift: float, drift_dt: float, kick_coef: float, pos_bar, vel_bar,
                        mass_bar, ws, opts: nb_opts):
    import torch
    f64 = torch.float64
    n = mass.shape[0]
    _check(lib().nb_step_vjp_reverse(
        _dptr(pos, "pos", f64), _dptr(vhalf, "vhalf", f64), _dptr(acc, "acc", f64),
        _dptr(mass, "mass", f64), n, float(eps), float(rewind_kick), float(rewind_drift),
        float(drift_dt), float(kick_coef), _dptr(pos_bar, "pos_bar", f64),
        _dptr(vel_bar, "vel_bar", f64), _dptr(mass_bar, "mass_bar", f64), _dptr(ws, "ws"),
        ws.numel() * ws.element_size(), ctypes.byref(opts)))


def nb_forces_jerk(pos, vel, mass, eps: float, acc, jerk, pot, ws, opts: nb_opts):
    import torch
    f64 = torch.float64
    n = mass.shape[0]
    _check(lib().nb_forces_jerk(
        _dptr(pos, "pos", f64), _dptr(vel, "vel", f64), _dptr(mass, "mass", f64), n, float(eps),
        _dptr(acc, "acc", f64), _dptr(jerk, "jerk", f64), _dptr(pot, "pot", f64, True),
        _dptr(ws, "ws"), ws.numel() * ws.element_size(), ctypes.byref(opts)))


def nb_hermite4(pos, vel, mass, eps: float, acc, jerk, acc_valid: bool, dt: float, nsteps: int,
                ws, opts: nb_opts):
    import torch
    f64 = torch.float64
    n = mass.shape[0]
    _check(lib().nb_hermite4(
        _dptr(pos, "pos", f64), _dptr(vel, "vel", f64), _dptr(mass, "mass", f64), n, float(eps),
        _dptr(acc, "acc", f64), _dptr(jerk, "jerk", f64), int(bool(acc_valid)), float(dt),
        int(nsteps), _dptr(ws, "ws"), ws.numel() * ws.element_size(), ctypes.byref(opts)))


def nb_poll_status(ws, opts: nb_opts | None = None) -> int:
    """Synchronises the stream and returns the latched device status code;
    ws=None polls nb_forces_noalloc's fixed array on the current device."""
    stream = opts.stream if opts is not None else None
    if ws is None:
        return int(lib().nb_poll_status(None, 0, stream))
    rc = lib().nb_poll_status(_dptr(ws, "ws"), ws.numel() * ws.element_size(), stream)
    return int(rc)


def make_state(pos, vel, mass, acc, pot, eps: float, ws, offsets=None, eps_b=None,
               acc_valid: bool = False) -> nb_state:
    """nb_state over caller-owned tensors (kept alive on the returned object)."""
    import torch
    f64 = torch.float64
    s = nb_state()
    s.N = mass.shape[0]
    s.B = 1 if offsets is None else offsets.shape[0] - 1
    s.offsets = _dptr(offsets, "offsets", torch.int64, True)
    s.pos = _dptr(pos, "pos", f64)
    s.vel = _dptr(vel, "vel", f64)
    s.mass = _dptr(mass, "mass", f64)
    s.acc = _dptr(acc, "acc", f64)
    s.pot = _dptr(pot, "pot", f64, True)
    s.eps_b = _dptr(eps_b, "eps_b", f64, True)
    s.eps = float(eps)
    s.step = 0
    s.acc_valid = int(bool(acc_valid))
    s.ws = _dptr(ws, "ws")
    s.ws_bytes = ws.numel() * ws.element_size()
    s._refs = (pos, vel, mass, acc, pot, ws, offsets, eps_b)
    return s
