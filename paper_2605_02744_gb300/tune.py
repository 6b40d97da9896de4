"""Launch-shape autotuner with a JSON cache.

For the single-system kernels a candidate is an nb_tune (threads, i-particles
per thread, j-tile, bulk-copy stages, persistent CTAs per SM); for batches it
is the work-item width in j-blocks (symmetric pairs, the default) or the
thread-block-cluster size (direct pairs).  Every candidate this
build compiled (``nb_tune_valid``) is timed on the caller's inputs with CUDA
events after a warm-up; the fastest median wins, ties going to the smaller
resource use.  Results are cached per (device name, compute capability,
kind, precision, N rounded up to a power of two) in
``$NB_TUNE_CACHE`` (default ``~/.cache/nbody_gb300/tune.json``).
"""
from __future__ import annotations

import json
import os
import statistics
import threading

import torch

from . import binding as B

_lock = threading.Lock()

FORCE_CANDIDATES = [
    dict(threads=t, i_per_thread=i, tile_j=j, stages=s, ctas_per_sm=c)
    for (t, i, j, s) in [(512, 2, 1024, 2), (512, 2, 512, 2), (256, 2, 512, 2), (256, 2, 256, 3),
                         (256, 4, 256, 3), (128, 2, 128, 3), (128, 1, 64, 2)]
    for c in (1, 2, 4)
]
BATCHED_CANDIDATES = [dict(cluster_ctas=c, threads=t) for c in (2, 4, 8) for t in (256, 512)]
BATCHED_SYM_CANDIDATES = [dict(item_blocks=g) for g in (2, 4, 8)]
VJP_CANDIDATES = [
    dict(threads=t, i_per_thread=i, tile_j=j, stages=s, ctas_per_sm=4)
    for (t, i, j, s) in [(128, 2, 128, 3), (256, 2, 128, 3), (256, 1, 128, 3), (128, 1, 64, 2)]
]


def cache_path() -> str:
    return os.environ.get("NB_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "nbody_gb300",
                                       "tune.json"))


def _bucket(n: int) -> int:
    b = 1
    while b < n:
        b <<= 1
    return b


def _key(kind: str, precision: str, n: int, device=None) -> str:
    props = torch.cuda.get_device_properties(device or torch.cuda.current_device())
    return f"{props.name}|sm{props.major}{props.minor}|{kind}|{precision}|N{_bucket(n)}"


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value: dict) -> None:
    with _lock:
        data = _load()
        data[key] = value
        path = cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def lookup(kind: str, precision: str, n: int):
    """The cached tune for this device/kind/precision/size bucket, or None."""
    hit = _load().get(_key(kind, precision, n))
    return None if hit is None else hit["tune"]


def _median_ms(fn, reps: int) -> float:
    st = torch.cuda.current_stream()
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def _cost(t: dict) -> tuple:
    # tie-break: fewer threads x i-per-thread, then fewer stages, then CTAs
    # (wider batched items: fewer records, less workspace)
    return (t.get("threads", 0) * t.get("i_per_thread", 0), t.get("stages", 0),
            t.get("ctas_per_sm", 0), t.get("cluster_ctas", 0), -t.get("item_blocks", 0))


def batched_pairs(precision: str, pairs: str = "default") -> str:
    """The pair path a batched call takes: "symmetric" unless direct pairs are
    asked for or the pairs are FP64 (which only the direct kernel computes)."""
    return "direct" if pairs == "direct" or precision == "fp64" else "symmetric"


def autotune_forces(pos, mass, eps: float, precision="kahan", reps: int = 5, warmup: int = 2,
                    candidates=None, store: bool = True) -> dict:
    """Time nb_forces for every compiled candidate; returns the best nb_tune dict.

    The candidates are shapes of the direct (every ordered pair) kernel, which
    is what is timed; the symmetric-pair path has one fixed shape.
    """
    n = mass.shape[0]
    acc = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
    pot = torch.empty(n, dtype=torch.float64, device=pos.device)
    results = []
    for cand in candidates or FORCE_CANDIDATES:
        if not B.nb_tune_valid(cand):
            continue
        opts = B.make_opts(precision, tune=cand, pairs="direct")
        ws = B.workspace(n, 1, opts, pos.device)
        run = lambda: B.nb_forces(pos, mass, eps, acc, pot, ws, opts)
        for _ in range(warmup):
            run()
        results.append((_median_ms(run, reps), _cost(cand), cand))
        del ws
    results.sort(key=lambda r: (r[0], r[1]))
    best = results[0]
    if store:
        _store(_key("force", precision, n),
               {"tune": best[2], "ms": best[0],
                "all": [{"tune": c, "ms": t} for t, _, c in results]})
    return best[2]


def autotune_batched(pos, vel, mass, offsets, eps, dt: float, nsteps: int = 20,
                     precision="f64acc", reps: int = 3, candidates=None,
                     store: bool = True, pairs: str = "default") -> dict:
    """Time nsteps batched KDK steps per candidate; returns the best nb_tune dict.

    The candidates are those of the path `pairs` resolves to (batched_pairs):
    the work-item width of the symmetric path, or the cluster size and CTA
    threads of the direct kernel.  The result is cached under the kind
    "batched-symmetric" or "batched-direct".
    """
    from .api import System
    n = mass.shape[0]
    path = batched_pairs(precision, pairs)
    default = BATCHED_SYM_CANDIDATES if path == "symmetric" else BATCHED_CANDIDATES
    results = []
    device = pos.device if torch.is_tensor(pos) else "cuda"
    for cand in candidates or default:
        # the trial runs step copies: the caller's state is left as it was
        sysm = System(torch.as_tensor(pos, dtype=torch.float64, device=device).clone(),
                      torch.as_tensor(vel, dtype=torch.float64, device=device).clone(), mass, eps,
                      offsets=offsets, precision=precision, tune=cand, device=device,
                      pairs=path)
        sysm.step(dt, 1)
        t = _median_ms(lambda: sysm.step(dt, nsteps), reps)
        results.append((t, _cost(cand), cand))
        del sysm
    results.sort(key=lambda r: (r[0], r[1]))
    best = results[0]
    if store:
        _store(_key("batched-" + path, precision, n),
               {"tune": best[2], "ms": best[0],
                "all": [{"tune": c, "ms": t} for t, _, c in results]})
    return best[2]
