"""CPU-only checks of the C ABI: the library loads, exports every entry point
declared in include/nbody.h, and rejects bad arguments on the host before
touching a device (no GPU is needed for any of these calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    import paper_2605_02744_gb300 as pkg
    pkg.build()
    from paper_2605_02744_gb300 import binding
    binding.lib()
    return binding


def _declared():
    src = open(os.path.join(ROOT, "include", "nbody.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(B):
    names = _declared()
    assert len(names) >= 13
    lib = B.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.EXPORTED) == names


def test_integer_fp_conversions_match_c(B):
    """The integer-pipe float <-> double conversions (round to nearest even
    for double -> float) and finiteness test of the FP64-bound batched fold
    give the IEEE results bit for bit."""
    assert B.nb_check_fp_conversions(300000, seed=1) == 0
    assert B.nb_check_fp_conversions(300000, seed=2) == 0
    with pytest.raises(B.NbError):
        B.nb_check_fp_conversions(-1)


def test_version_and_defaults(B):
    assert "sm_103a" in B.nb_version()
    o = B.nb_opts()
    B.lib().nb_opts_default(ctypes.byref(o))
    assert o.precision == B.NB_PREC_F64ACC and o.G == 1.0 and o.stream is None
    assert o.use_graph == 0 and not o.tune and o.timeout_cycles == 0


def _opts(B, **kw):
    o = B.nb_opts()
    B.lib().nb_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def test_workspace_sizes(B):
    o = _opts(B)
    assert B.nb_workspace_bytes(0, 1, o) == 0
    assert B.nb_workspace_bytes(10, 0, o) == 0
    sizes = [B.nb_workspace_bytes(n, 1, o) for n in (1, 1000, 100000, 1 << 20)]
    assert all(s % 256 == 0 for s in sizes)
    assert sizes == sorted(sizes)
    # the packed copy alone needs 32 B per (padded) particle
    assert sizes[-1] >= 32 * (1 << 20)


def test_tune_validation(B):
    assert B.nb_tune_valid({"threads": 256, "i_per_thread": 4, "tile_j": 256, "stages": 3})
    assert B.nb_tune_valid({"threads": 512, "i_per_thread": 2, "tile_j": 1024, "stages": 2})
    assert B.nb_tune_valid({"threads": 128, "i_per_thread": 1, "tile_j": 64, "stages": 2})
    assert not B.nb_tune_valid({"threads": 96, "i_per_thread": 4, "tile_j": 256, "stages": 3})
    assert not B.nb_tune_valid({"threads": 256, "i_per_thread": 4, "tile_j": 256, "stages": 3,
                                "ctas_per_sm": 9})


FAKE = 1 << 20  # an aligned non-NULL address; never dereferenced by these calls


def _forces(B, N=16, eps=0.1, pos=FAKE, mass=FAKE, acc=FAKE, pot=None, ws=FAKE, wsb=None,
            opts=None):
    opts = opts or _opts(B)
    if wsb is None:
        wsb = B.nb_workspace_bytes(max(N, 1), 1, opts)
    return B.lib().nb_forces(pos, mass, N, eps, acc, pot, ws, wsb, ctypes.byref(opts))


@pytest.mark.parametrize("kw,code", [
    ({"N": 0}, 1), ({"N": -5}, 1), ({"eps": -1.0}, 1), ({"eps": float("nan")}, 1),
    ({"eps": float("inf")}, 1), ({"eps": 1e-30}, 1), ({"pos": None}, 1), ({"mass": None}, 1),
    ({"acc": None}, 1), ({"pos": FAKE + 4}, 1), ({"pot": FAKE + 2}, 1), ({"ws": None}, 1),
    ({"ws": FAKE + 16}, 1), ({"wsb": 1024}, 3),
])
def test_nb_forces_rejects_bad_arguments(B, kw, code):
    assert _forces(B, **kw) == code
    assert B.nb_last_error() != ""


def test_bad_opts(B):
    assert _forces(B, opts=_opts(B, precision=7)) == B.NB_ERR_INVALID
    assert _forces(B, opts=_opts(B, G=float("inf"))) == B.NB_ERR_INVALID
    assert _forces(B, opts=_opts(B, timeout_cycles=-1)) == B.NB_ERR_INVALID
    bad = B.nb_tune(threads=96, i_per_thread=4, tile_j=256, stages=3, ctas_per_sm=1)
    o = _opts(B)
    o.tune = ctypes.pointer(bad)
    assert _forces(B, opts=o) == B.NB_ERR_UNSUPPORTED
    assert B.lib().nb_forces(FAKE, FAKE, 16, 0.1, FAKE, None, FAKE, 1 << 30, None) == 1


def test_step_and_vjp_argument_checks(B):
    o = _opts(B)
    st = B.nb_state()
    st.N, st.B = 16, 1
    st.pos = st.vel = st.mass = st.acc = FAKE
    st.ws, st.ws_bytes = FAKE, B.nb_workspace_bytes(16, 1, o)
    lib = B.lib()
    assert lib.nb_step(None, 1e-3, 1, ctypes.byref(o)) == 1
    assert lib.nb_step(ctypes.byref(st), float("nan"), 1, ctypes.byref(o)) == 1
    assert lib.nb_step(ctypes.byref(st), 1e-3, -1, ctypes.byref(o)) == 1
    st.vel = None
    assert lib.nb_step(ctypes.byref(st), 1e-3, 1, ctypes.byref(o)) == 1
    st.vel = FAKE
    st.B = 4  # batched without offsets
    assert lib.nb_step(ctypes.byref(st), 1e-3, 1, ctypes.byref(o)) == 1
    wsb = st.ws_bytes
    assert lib.nb_forces_vjp(FAKE, FAKE, 16, 0.1, None, None, FAKE, FAKE, FAKE, wsb,
                             ctypes.byref(o)) == 1
    assert lib.nb_step_vjp(FAKE, FAKE, 16, 0.1, float("inf"), 0.5, FAKE, FAKE, FAKE, FAKE, wsb,
                           ctypes.byref(o)) == 1
    assert lib.nb_step_vjp(FAKE, FAKE, 16, 0.1, 1e-3, 5e-4, FAKE, None, FAKE, FAKE, wsb,
                           ctypes.byref(o)) == 1
    # row ranges: a bad range, a non-finite coefficient, a missing cotangent
    for i0, i1 in ((-1, 4), (4, 4), (0, 17)):
        assert lib.nb_forces_range(FAKE, FAKE, 16, i0, i1, 0.1, FAKE, None, FAKE, wsb,
                                   ctypes.byref(o)) == 1
        assert lib.nb_forces_vjp_range(FAKE, FAKE, 16, i0, i1, 0.1, 1.0, FAKE, None, FAKE, FAKE,
                                       FAKE, wsb, ctypes.byref(o)) == 1
    assert lib.nb_forces_vjp_range(FAKE, FAKE, 16, 0, 8, 0.1, float("nan"), FAKE, None, FAKE,
                                   FAKE, FAKE, wsb, ctypes.byref(o)) == 1
    assert lib.nb_forces_vjp_range(FAKE, FAKE, 16, 0, 8, 0.1, 1.0, None, None, FAKE, FAKE, FAKE,
                                   wsb, ctypes.byref(o)) == 1
    assert lib.nb_kick_drift(FAKE, FAKE, FAKE, 0, 0.5, 1.0, ctypes.byref(o)) == 1
    assert lib.nb_kick_drift(FAKE, FAKE, FAKE, 4, float("inf"), 1.0, ctypes.byref(o)) == 1
    assert lib.nb_forces_batched(FAKE, FAKE, FAKE, 0, 16, FAKE, FAKE, None, FAKE, 1 << 30,
                                 ctypes.byref(o)) == 1
    assert lib.nb_forces_batched(FAKE, FAKE, FAKE, 4, 3, FAKE, FAKE, None, FAKE, 1 << 30,
                                 ctypes.byref(o)) == 1
    assert lib.nb_energy(ctypes.byref(st), None, ctypes.byref(o)) == 1
    # a workspace of fewer than 256 bytes is refused before any device call;
    # NULL names nb_forces_noalloc's fixed array, which needs a device
    assert lib.nb_poll_status(FAKE, 255, None) == 1
    assert lib.nb_poll_status(None, 0, None) in (0, 2)


def test_python_binding_requires_cuda_tensors(B):
    import torch
    o = _opts(B)
    x = torch.zeros((4, 3), dtype=torch.float64)
    with pytest.raises(TypeError):
        B.nb_forces(x, x[:, 0].contiguous(), 0.1, x, None, torch.zeros(256, dtype=torch.uint8), o)


def test_pairs_option_and_symmetric_workspace(B):
    o = _opts(B)
    assert o.pairs == B.NB_PAIRS_DEFAULT
    n = 1 << 20
    nb = n // 2048
    default = B.nb_workspace_bytes(n, 1, o)
    direct = B.nb_workspace_bytes(n, 1, _opts(B, pairs=B.NB_PAIRS_DIRECT))
    # the symmetric path adds O(N) scratch: 64 B of fixed-point totals per
    # slot plus 12 B of cost estimates per block pair
    extra = default - direct
    assert 64 * n <= extra <= 64 * n + 12 * nb * (nb + 1) // 2 + 64 * 1024
    assert default <= 512 << 20
    n4 = 1 << 22
    extra4 = (B.nb_workspace_bytes(n4, 1, o)
              - B.nb_workspace_bytes(n4, 1, _opts(B, pairs=B.NB_PAIRS_DIRECT)))
    assert extra4 <= 4.5 * extra
    # below the default range only an explicit request provisions the path
    small_default = B.nb_workspace_bytes(1000, 1, o)
    small_sym = B.nb_workspace_bytes(1000, 1, _opts(B, pairs=B.NB_PAIRS_SYMMETRIC))
    assert small_sym > small_default
    # FP64 pairs use the same fixed-point totals; above 2^24 the default is
    # the direct kernel
    fp64 = _opts(B, precision=B.NB_PREC_FP64)
    fp64_direct = _opts(B, precision=B.NB_PREC_FP64, pairs=B.NB_PAIRS_DIRECT)
    assert B.nb_workspace_bytes(n, 1, fp64) - B.nb_workspace_bytes(n, 1, fp64_direct) == extra
    above = (1 << 24) + 2048
    assert B.nb_workspace_bytes(above, 1, o) == \
        B.nb_workspace_bytes(above, 1, _opts(B, pairs=B.NB_PAIRS_DIRECT))


def test_unknown_pairs_mode_is_rejected(B):
    rc = _forces(B, opts=_opts(B, pairs=7))
    assert rc == B.NB_ERR_INVALID


def test_batched_symmetric_workspace(B):
    # batches (B > 1) provision the symmetric batched region unless pairs is
    # DIRECT or the policy is FP64; it grows with N + 128 B (padded slots)
    n, b = 100000, 64
    sym = B.nb_workspace_bytes(n, b, _opts(B))
    direct = B.nb_workspace_bytes(n, b, _opts(B, pairs=B.NB_PAIRS_DIRECT))
    fp64 = B.nb_workspace_bytes(n, b, _opts(B, precision=B.NB_PREC_FP64))
    assert sym > direct and fp64 == direct
    slots = n + 128 * b
    assert sym - direct >= 2 * 80 * slots  # two slot-order FP64 state buffers
    assert B.nb_workspace_bytes(2 * n, b, _opts(B)) > sym


def test_batched_item_width(B):
    # nb_tune.item_blocks: 2, 4 or 8 j-blocks per symmetric batched work item
    # (0 = 8); each item owns a 4 KiB FP64 record, provisioned for 18, 10 or
    # 6 items per 128-slot block
    for g in (0, 2, 4, 8):
        assert B.nb_tune_valid({"item_blocks": g})
    for g in (1, 3, 16, -2):
        assert not B.nb_tune_valid({"item_blocks": g})
    n, b = 100000, 64
    blocks = -(-(n + 128 * b) // 128)

    def ws(g):
        t = B.nb_tune(item_blocks=g)
        o = _opts(B, tune=ctypes.pointer(t))
        return B.nb_workspace_bytes(n, b, o)

    assert ws(0) == ws(8) == B.nb_workspace_bytes(n, b, _opts(B))
    assert ws(4) - ws(8) >= 4 * blocks * 4096
    assert ws(2) - ws(8) >= 12 * blocks * 4096
    # the direct path ignores the field
    t = B.nb_tune(item_blocks=2)
    d = _opts(B, pairs=B.NB_PAIRS_DIRECT, tune=ctypes.pointer(t))
    assert B.nb_workspace_bytes(n, b, d) == B.nb_workspace_bytes(
        n, b, _opts(B, pairs=B.NB_PAIRS_DIRECT))


def test_kernel_timing_hook_without_launches(B):
    lib = B.lib()
    assert lib.nb_kernel_timing(1) == B.NB_OK
    assert B.nb_kernel_time() == (0.0, 0)
    assert lib.nb_kernel_time(None, None) == B.NB_ERR_INVALID
    assert lib.nb_kernel_timing(0) == B.NB_OK
