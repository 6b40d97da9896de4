#!/usr/bin/env python
"""Benchmark of the direct N-body hot path on GB300.

Metric: G pair-interactions/s on a 2^20-particle Plummer sphere (eps = 1e-3,
FP32 pairs with Kahan-compensated accumulation), one step = one kick-drift-kick
leapfrog step through nb_step (kick + drift, Hilbert-sorted FP32 pack, the
all-pairs force + potential evaluation, its fold with the closing half-kick)
followed by nb_energy.  Interactions are counted as N^2 per step, the
metric's convention; the default symmetric-pair path evaluates each
unordered pair once and applies it to both particles (Newton's third law),
the direct path (timed alongside) every ordered pair.  Alongside: the
FP64-accumulate variant's rate, the adjoint/forward time ratio of the
16384-particle, 200-step gradient, the roofline of the step against the FP32
FMA peak (20 flops per interaction), the end-to-end rate from host buffers,
and the FP64 oracle timed on the host cores on a sample of rows; on those
exact rows, the relative errors of each timed configuration's forces at the
initial positions ("accuracy": gated at 1e-5 in the tests).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank advances its own replica of the 2^20 step
(weak scaling, no data exchange), value = all ranks' interactions / max
time; the "sharded" object beside it times the same system split over the
ranks by rows (strong scaling: nb_forces_range per rank, one NCCL
all-gather of the positions per step), also at N = 1 as its baseline.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G pair-interactions/s at N=2^20 vs FP32 roofline; adjoint/forward time at 1e-5 err"
UNIT = "G pair-interactions/s"
N_MAIN = 1 << 20
EPS_MAIN = 1e-3
DT_MAIN = 1e-4
FLOPS_PER_INTERACTION = 20
FP32_LANES_PER_SM = 128
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "force_sym_plummer_2p20_traffic.txt")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device):
    """Max of a per-rank number over all ranks of the process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world: int, steps: int, interactions_per_step: float, max_ms: float) -> float:
    """Whole-job rate: every rank's interactions over the slowest rank's time
    (replicas, weak scaling), in G interactions/s."""
    return world * steps * interactions_per_step / (max_ms * 1e-3) / 1e9


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix=f"nb_clocks_gpu{index}_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            try:
                os.unlink(self.path)
            except OSError:
                pass
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9 and p[1].replace(".", "").isdigit():
                    rows.append(p)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        load = [float(r[1]) for r in rows if float(r[3]) > 200.0] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


def _kernel_source_hash():
    """Hash of the pair kernel's source: the device code of nb_sym.cu (from
    its constants to the end of force_sym_kernel, host launch code excluded)
    and the device headers it includes."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2605_02744_gb300", "csrc")
    h = hashlib.sha256()
    with open(os.path.join(csrc, "nb_sym.cu")) as fh:
        src = fh.read()
    a = src.index("constexpr int BI = 2048;")
    b = src.index("__global__ void __launch_bounds__(256) sym_fold_kernel(")
    h.update(src[a:b].encode())
    for f in ("nb_symj.cuh", "nb_sym_core.cuh", "nb_device.cuh", "nb_fixed.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic():
    """DRAM bytes per force launch from the committed ncu summary, or None
    when the kernel source changed after the counters were taken."""
    vals = {}
    try:
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.strip()
    except OSError:
        return None
    if vals.get("source_sha256_16") != _kernel_source_hash():
        return None
    return float(vals["dram_bytes_per_launch"]) if "dram_bytes_per_launch" in vals else None


def cpu_baseline(seconds: float = 10.0, gpu=None, gpu65536=None):
    """FP64 oracle rows on the host cores: exact a_i, phi_i for sampled i.

    `gpu`: {name: (acc [N, 3], pot [N])} from GPU evaluations at the same
    positions; their errors on the sampled rows are returned as a second
    value (see accuracy_on_rows).  `gpu65536`: the same for the 65536
    log-normal workload's precision variants, compared with the rows the
    oracle computes for its rate on that workload."""
    import numpy as np

    import oracle
    from paper_2605_02744_gb300 import ics
    oracle.build()
    s = ics.plummer(N_MAIN, seed=0)
    rng = np.random.default_rng(4)
    t0 = time.perf_counter()
    probe = rng.choice(N_MAIN, 64, replace=False)
    oracle.forces_rows(s.pos, s.mass, EPS_MAIN, probe)
    dt = time.perf_counter() - t0
    nrows = int(max(64, min(N_MAIN, 64 * seconds / max(dt, 1e-3))))
    rows = rng.choice(N_MAIN, nrows, replace=False)
    t0 = time.perf_counter()
    ra, rp = oracle.forces_rows(s.pos, s.mass, EPS_MAIN, rows)
    el = time.perf_counter() - t0
    rate = nrows * N_MAIN / el / 1e9
    info = {"value": rate, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{nrows} exact rows x {N_MAIN} j of the 2^20 Plummer sphere "
                      f"(FP64 C, OpenMP over rows), {el:.1f} s",
            }
    info["other_sizes"], exact = _oracle_other_sizes()
    acc = None
    if gpu:
        acc = {"rows": nrows, "reference": "the FP64 oracle's exact rows above",
               "gate": 1e-5}
        for name, (a, p) in gpu.items():
            acc[name] = accuracy_on_rows(a[rows], p[rows], ra, rp)
    if gpu65536 and acc is not None:
        r65, ra65, rp65 = exact["plummer_lognormal_65536"]
        acc["lognormal_65536"] = {
            "rows": int(r65.shape[0]),
            "reference": "the oracle's exact rows of other_sizes.plummer_lognormal_65536",
            "gates_in_tests": {"f64acc": 1e-5, "kahan": 1e-5, "fp64": 1e-12,
                               "fp32": "none (single-float displacements)"},
            **{name: accuracy_on_rows(a[r65], p[r65], ra65, rp65)
               for name, (a, p) in gpu65536.items()}}
    return info, acc


def _oracle_other_sizes(seconds: float = 2.0):
    """The oracle's rate on the 65536 log-normal and 16384 Plummer workloads
    (sampled rows against all j, about `seconds` each), for comparison, and
    those exact rows ({name: (rows, acc, pot)})."""
    import numpy as np

    import oracle
    from paper_2605_02744_gb300 import ics
    out, exact = {}, {}
    for name, s, eps in (("plummer_lognormal_65536", ics.plummer_lognormal(65536, 0), 1e-3),
                         ("plummer_16384", ics.plummer(16384, 0), 5e-3)):
        n = s.mass.shape[0]
        rng = np.random.default_rng(4)
        t0 = time.perf_counter()
        oracle.forces_rows(s.pos, s.mass, eps, rng.choice(n, 256, replace=False))
        dt = time.perf_counter() - t0
        nrows = int(max(256, min(n, 256 * seconds / max(dt, 1e-3))))
        rows = rng.choice(n, nrows, replace=False)
        t0 = time.perf_counter()
        ra, rp = oracle.forces_rows(s.pos, s.mass, eps, rows)
        el = time.perf_counter() - t0
        out[name] = {"value": nrows * n / el / 1e9, "unit": UNIT, "rows": nrows}
        exact[name] = (rows, ra, rp)
    return out, exact


def accuracy_on_rows(a, p, ra, rp):
    """Relative errors of GPU (a, p) against exact rows (ra, rp): per particle
    |a - a_ref| / |a_ref| (vector norm; gated at 1e-5) and |p - p_ref| / |p_ref|
    as max, 99.9th percentile and median; also the component-wise relative
    deviation (the paper's form, ill-conditioned where a component is near
    zero) as median and 99th percentile."""
    import numpy as np
    e = np.linalg.norm(a - ra, axis=1) / np.linalg.norm(ra, axis=1)
    ep = np.abs(p - rp) / np.abs(rp)
    ec = (np.abs(a - ra) / np.abs(ra)).ravel()
    return {"acc_max": float(e.max()), "acc_p999": float(np.quantile(e, 0.999)),
            "acc_median": float(np.median(e)), "pot_max": float(ep.max()),
            "pot_median": float(np.median(ep)),
            "componentwise_median": float(np.median(ec)),
            "componentwise_p99": float(np.quantile(ec, 0.99)),
            "pass": bool(e.max() <= 1e-5 and ep.max() <= 1e-5)}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_2605_02744_gb300 import ics
    oracle.build()
    s = ics.plummer(N_MAIN, seed=0)
    rng = np.random.default_rng(4)
    rows_per_step = 512
    for _ in range(args.warmup):
        oracle.forces_rows(s.pos, s.mass, EPS_MAIN, rng.choice(N_MAIN, rows_per_step, False))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.forces_rows(s.pos, s.mass, EPS_MAIN, rng.choice(N_MAIN, rows_per_step, False))
    el = time.perf_counter() - t0
    value = args.steps * rows_per_step * N_MAIN / el / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Plummer N=2^20, eps=1e-3, force+potential rows "
                                   f"({rows_per_step} sampled i x all j per step)",
                       "N": N_MAIN},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{rows_per_step} exact rows per step x {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_steps(system, dt, steps, flush, torch):
    """Per-step CUDA-event times (ms) on the library's stream, L2 flushed in between."""
    st = torch.cuda.current_stream()
    times = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        system.step(dt, 1)
        system.energy()
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def batched_rate(torch, steps=1000):
    """512 independent Plummer clusters (N_c log-uniform 64..8192, eps 0.01),
    `steps` KDK steps dt=1e-3 replayed as one CUDA graph: the symmetric-pair
    batched path (each unordered pair of a cluster once), its work-item width
    picked by the autotuner on 20-step runs of the same workload (untimed)."""
    import numpy as np

    from paper_2605_02744_gb300 import api, ics, tune
    s = ics.batched_plummer(512, seed=1)
    sizes = np.diff(s.offsets).astype(np.float64)
    eps = np.full(512, 0.01)
    best = tune.autotune_batched(torch.tensor(s.pos, device="cuda"),
                                 torch.tensor(s.vel, device="cuda"),
                                 torch.tensor(s.mass, device="cuda"), s.offsets, eps, 1e-3,
                                 nsteps=20, reps=3, store=False)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        g = api.System(s.pos, s.vel, s.mass, eps, offsets=s.offsets, precision="f64acc",
                       stream=st, use_graph=True, tune=best)
        g.forces()
        g.step(1e-3, steps)  # first call captures the step loop as a graph
        g.pos.copy_(torch.tensor(s.pos, device="cuda"))
        g.vel.copy_(torch.tensor(s.vel, device="cuda"))
        g.forces()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        g.step(1e-3, steps)  # graph replay
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        ok = g.poll()
    inter = float((sizes ** 2).sum()) * steps
    return {"workload": f"512 Plummer clusters, N_c log-uniform [64, 8192] (seed 1), "
                        f"eps=0.01, {steps} KDK steps dt=1e-3, F64ACC, symmetric pairs "
                        f"(warp-granular items, per-cluster Hilbert order), one CUDA graph",
            "ms": ms, "value": inter / (ms * 1e-3) / 1e9, "unit": UNIT, "status": ok,
            "interactions": inter, "tune": best}


def batched_sharded_rate(torch, ws, dev, tune, steps=1000):
    """The 512-cluster workload split over the ranks by cluster (strong
    scaling: the same batch on every N; clusters go largest first to the
    least-loaded rank, and nothing is exchanged while they step): each rank
    replays its own clusters' 1000-step CUDA graph; max over ranks of the
    CUDA-event time; the rate counts every cluster's pairs."""
    import numpy as np

    from paper_2605_02744_gb300 import ics
    from paper_2605_02744_gb300.sharded import ShardedBatch
    s = ics.batched_plummer(512, seed=1)
    sizes = np.diff(s.offsets).astype(np.float64)
    eps = np.full(512, 0.01)
    st = torch.cuda.Stream(dev)
    with torch.cuda.stream(st):
        g = ShardedBatch(s.pos, s.vel, s.mass, s.offsets, eps, precision="f64acc", device=dev,
                         stream=st, use_graph=True, tune=tune)
        if g.ops is not None:
            sysm = g.ops.sys
            sysm.forces()
            sysm.step(1e-3, steps)  # first call captures the step loop as a graph
            sysm.pos.copy_(torch.tensor(s.pos[g.rows], device=dev))
            sysm.vel.copy_(torch.tensor(s.vel[g.rows], device=dev))
            sysm.forces()
        st.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        g.step(1e-3, steps)  # graph replay
        e1.record(st)
        e1.synchronize()
    ms = e0.elapsed_time(e1)
    ok = g.ops.poll() if g.ops is not None else 0
    if ws > 1:
        ms = max_over_ranks(ms, dev)
    inter = float((sizes ** 2).sum()) * steps
    return {"workload": f"the 512-cluster batch split over {ws} rank(s) by cluster "
                        f"(no data exchange), {steps} KDK steps dt=1e-3 in one CUDA graph "
                        f"per rank, F64ACC, symmetric pairs",
            "scaling": "strong", "n_gpus": ws, "clusters_on_rank0": len(g.clusters),
            "ms": ms, "value": inter / (ms * 1e-3) / 1e9, "unit": UNIT, "status": ok}


def paper_workload(torch):
    """The paper's benchmark size (Sec. 4.2): 409600 particles, 3 steps of a
    Hermite scheme with acceleration + jerk (here fourth order; the paper's is
    sixth order and runs its predictor/corrector on the host).  Context for
    its Table 1, not a like-for-like comparison."""
    from paper_2605_02744_gb300 import binding, ics
    n, steps, eps, dt = 409600, 3, 1e-3, 1e-3
    s = ics.plummer(n, seed=0)
    o = binding.make_opts("kahan")
    pos = torch.tensor(s.pos, device="cuda")
    vel = torch.tensor(s.vel, device="cuda")
    mass = torch.tensor(s.mass, device="cuda")
    acc = torch.empty_like(pos)
    jerk = torch.empty_like(pos)
    ws = binding.workspace(n, 1, o)
    binding.nb_hermite4(pos, vel, mass, eps, acc, jerk, False, dt, 1, ws, o)  # warm-up
    pos.copy_(torch.tensor(s.pos, device="cuda"))
    vel.copy_(torch.tensor(s.vel, device="cuda"))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    binding.nb_hermite4(pos, vel, mass, eps, acc, jerk, False, dt, steps, ws, o)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    evals = steps + 1
    return {"workload": "Plummer N=409600, eps=1e-3, 3 Hermite-4 steps dt=1e-3 "
                        "(acceleration + jerk, FP32 pairs, Kahan), including the first "
                        "evaluation", "seconds": ms / 1e3,
            "acc_jerk_interactions_per_s": evals * float(n) * n / (ms * 1e-3),
            "paper_seconds": {"wormhole_n300_1chip": 1459.46,
                              "cpu_2x_epyc9124_32threads": 2875.39},
            "note": "paper: sixth-order Hermite, host FP64 predictor/corrector, whole run"}


def variant_rates(torch):
    """The 65536-particle log-normal workload: 10 KDK steps dt=1e-4 per
    precision variant (nb_step loop, energy not included).  Also returns
    each variant's forces at the initial positions (untimed), which the
    oracle leg compares with its exact rows."""
    from paper_2605_02744_gb300 import api, ics
    s = ics.plummer_lognormal(65536, seed=0)
    out = {"workload": "Plummer N=65536, log-normal masses (sigma 0.5), eps=1e-3, "
                       "10 KDK steps dt=1e-4"}
    first = {}
    for prec in ("f64acc", "kahan", "fp32", "fp64"):
        g = api.System(s.pos, s.vel, s.mass, 1e-3, precision=prec)
        g.forces()
        first[prec] = (g.acc.cpu().numpy(), g.pot.cpu().numpy())
        g.step(1e-4, 1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.step(1e-4, 10)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out[prec] = {"ms_10_steps": ms, "value": 10 * 65536.0 ** 2 / (ms * 1e-3) / 1e9}
    return out, first


def adjoint_ratio(torch):
    """Forward (200 KDK steps) vs gradient time at the 16384-particle workload;
    the target is the final state of an FP64-pair run (this library) from
    the initial positions perturbed by N(0, (1e-3)^2), seed 2."""
    from paper_2605_02744_gb300 import adjoint, api, ics
    s = ics.plummer(16384, seed=0)
    t = api.System(ics.perturb_positions(s.pos, 1e-3, seed=2), s.vel, s.mass, 5e-3,
                   precision="fp64")
    t.step(1e-3, 200)
    target = t.pos.cpu().numpy()
    del t
    return adjoint.time_forward_backward(s, target, eps=5e-3, dt=1e-3, nsteps=200, segment=20,
                                         precision="f64acc")


def sharded_rate(torch, args, ws, dev):
    """The 2^20 workload with its rows split over the ranks (strong scaling:
    the same system on every N): contiguous particle ranges, one position
    all-gather per step (NCCL), nb_forces_range for each rank's rows (the
    direct kernel) and the kick / drift of the rows; max over ranks of the
    CUDA-event time of the timed steps."""
    from paper_2605_02744_gb300 import ics
    from paper_2605_02744_gb300.sharded import ShardedSystem
    s = ics.plummer(N_MAIN, seed=0)
    g = ShardedSystem(s.pos, s.vel, s.mass, EPS_MAIN, precision="kahan", device=dev)
    for _ in range(args.warmup):
        g.step(DT_MAIN, 1)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    g.step(DT_MAIN, args.steps)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    if ws > 1:
        ms = max_over_ranks(ms, dev)
    return {"workload": "Plummer N=2^20, eps=1e-3, KDK steps dt=1e-4, rows split over "
                        f"{ws} rank(s) in contiguous ranges (Kahan, direct kernel per rank, "
                        "one FP64 position all-gather per step)",
            "scaling": "strong", "n_gpus": ws, "steps": args.steps,
            "ms_per_step": ms / args.steps,
            "value": args.steps * float(N_MAIN) ** 2 / (ms * 1e-3) / 1e9, "unit": UNIT,
            "rows_per_rank": g.c, "status": g.ops.poll()}


def run_ours(args):
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    import paper_2605_02744_gb300 as pkg
    from paper_2605_02744_gb300 import api, binding, ics
    pkg.build()
    s = ics.plummer(N_MAIN, seed=0)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    results = {}
    first = {}  # each configuration's forces at the initial positions (untimed)
    for prec, pairs in (("kahan", "default"), ("f64acc", "default"), ("kahan_direct", "direct")):
        if prec == "kahan_direct" and args.skip_extra:
            continue
        system = api.System(s.pos, s.vel, s.mass, EPS_MAIN, precision=prec.split("_")[0],
                            device=dev, pairs=pairs)
        system.forces()
        first[prec] = (system.acc.cpu().numpy(), system.pot.cpu().numpy())
        for _ in range(args.warmup):
            system.step(DT_MAIN, 1)
            system.energy()
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        n0 = binding.nb_launch_count()
        # the pair kernel's own launches, timed by CUDA events the library
        # records on its stream around each of them
        binding.nb_kernel_timing(True)
        with ClockSampler(dev.index or 0) as clk:
            times = _time_steps(system, DT_MAIN, args.steps, flush, torch)
        torch.cuda.synchronize()
        launches = binding.nb_launch_count() - n0
        try:
            kernel = binding.nb_kernel_time()
        except binding.NbError as e:
            kernel = str(e)
        binding.nb_kernel_timing(False)
        assert system.poll() == binding.NB_OK
        results[prec] = (times, clk.summary(), launches, kernel)
        del system
        torch.cuda.empty_cache()

    times, clocks, kahan_launches, kahan_kernel = results["kahan"]
    total_ms = sum(times)
    if ws > 1:
        total_ms = max_over_ranks(total_ms, dev)
        torch.distributed.barrier()
    inter = float(N_MAIN) * N_MAIN
    value = aggregate_rate(ws, args.steps, inter, total_ms)

    # end to end through the public API from pinned host buffers: every step
    # copies the state in (positions, velocities, masses and the previous
    # step's accelerations, so the step does the same work as a timed step:
    # one force + potential evaluation), runs nb_step(1) and nb_energy, and
    # copies positions, velocities, accelerations, potentials and energies out
    e2e_sys = api.System(s.pos, s.vel, s.mass, EPS_MAIN, precision="kahan", device=dev)
    e2e_sys.forces()
    host = {k: torch.as_tensor(getattr(s, k)).pin_memory() for k in ("pos", "vel", "mass")}
    host["acc"] = e2e_sys.acc.cpu().pin_memory()
    outs = {k: torch.empty(v.shape, dtype=torch.float64, pin_memory=True)
            for k, v in (("pos", e2e_sys.pos), ("vel", e2e_sys.vel), ("acc", e2e_sys.acc),
                         ("pot", e2e_sys.pot))}
    eh = torch.empty(3, dtype=torch.float64, pin_memory=True)
    st = torch.cuda.current_stream()

    def e2e_step():
        for k in ("pos", "vel", "mass", "acc"):
            getattr(e2e_sys, k).copy_(host[k], non_blocking=True)
        e2e_sys.state.acc_valid = 1
        e2e_sys.step(DT_MAIN, 1)
        eh.copy_(e2e_sys.energy(), non_blocking=True)
        for k in ("pos", "vel", "acc", "pot"):
            outs[k].copy_(getattr(e2e_sys, k), non_blocking=True)
        st.synchronize()

    e2e_step()
    e2e_steps = args.steps
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_el = time.perf_counter() - t0
    if ws > 1:  # the slowest rank's wall clock, as for the device-timed value
        e2e_el = max_over_ranks(e2e_el * 1e3, dev) * 1e-3
    e2e_value = ws * e2e_steps * inter / e2e_el / 1e9
    h2d = sum(v.numel() * 8 for v in host.values())
    d2h = sum(v.numel() * 8 for v in outs.values()) + 24
    del e2e_sys

    adj = batched = variants = paper = sharded = first65536 = None
    if not args.skip_extra:
        try:
            sharded = sharded_rate(torch, args, ws, dev)
        except Exception as e:
            sharded = {"error": f"{type(e).__name__}: {e}"}
    if not args.skip_adjoint:
        try:
            adj = adjoint_ratio(torch)
        except Exception as e:  # reported, never silently replaced
            adj = {"error": f"{type(e).__name__}: {e}"}
    batched_sharded = None
    if not args.skip_extra:
        try:
            batched = batched_rate(torch)
        except Exception as e:
            batched = {"error": f"{type(e).__name__}: {e}"}
        if ws > 1:  # on one GPU this is the batched leg itself
            try:
                batched_sharded = batched_sharded_rate(
                    torch, ws, dev, batched.get("tune") if isinstance(batched, dict) else None)
            except Exception as e:
                batched_sharded = {"error": f"{type(e).__name__}: {e}"}
        try:
            variants, first65536 = variant_rates(torch)
        except Exception as e:
            variants = {"error": f"{type(e).__name__}: {e}"}
        try:
            paper = paper_workload(torch)
        except Exception as e:
            paper = {"error": f"{type(e).__name__}: {e}"}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    peaks = _peaks()
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    step_ms = statistics.mean(times)
    achieved_step = FLOPS_PER_INTERACTION * inter / (step_ms * 1e-3) / 1e12
    if isinstance(kahan_kernel, tuple) and kahan_kernel[1] == args.steps:
        kernel_ms = kahan_kernel[0] / kahan_kernel[1]
        achieved = FLOPS_PER_INTERACTION * inter / (kernel_ms * 1e-3) / 1e12
        timing = ("CUDA events recorded by the library on the launch stream around each "
                  "force_sym_kernel launch of the timed steps (nb_kernel_timing)")
    else:  # the hook failed or saw another launch count: the whole step instead
        kernel_ms = None
        achieved = achieved_step
        timing = (f"kernel timing unavailable ({kahan_kernel}); CUDA events around each "
                  "whole nb_step+nb_energy instead")
    obs = clocks.get("sm_mhz")
    traffic = _traffic()
    if batched and "value" in batched:
        batched["frac_of_fp32_peak"] = FLOPS_PER_INTERACTION * batched["value"] / 1e3 / peak_tflops
    f64_ms = statistics.mean(results["f64acc"][0])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "Plummer sphere N=2^20 (1048576), equal mass, seed 0, eps=1e-3; "
                               "one KDK step dt=1e-4 (FP32 pairs, each unordered pair "
                               "evaluated once, Kahan accumulation, adaptive hi/lo "
                               "displacement, FP64 state) + energy",
                   "N": N_MAIN, "precision": "kahan", "interactions_per_step": "N^2",
                   "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                     "kernel": "force_sym_kernel<KAHAN, adaptive>",
                     "kernel_ms_per_launch": kernel_ms,
                     "frac_whole_step": achieved_step / peak_tflops,
                     "flops_per_interaction": FLOPS_PER_INTERACTION,
                     "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                   f"{max_mhz:.0f} MHz (max SM clock)",
                     "frac_at_observed_clock": (achieved / (peak_tflops * obs / max_mhz)
                                                if obs else None),
                     "timing": timing},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "how": "pinned host pos/vel/mass/acc -> device, nb_step (1 KDK step: one "
                       "force + potential evaluation), nb_energy, pos/vel/acc/pot/energy -> "
                       "host; wall clock"},
        "gpu_launches": kahan_launches,
        # the same rate with N (N - 1) interactions per step (no self pairs)
        "value_counting_n_n_minus_1": value * (N_MAIN - 1) / N_MAIN,
        "variants": {"f64acc_value": ws * args.steps * inter / (sum(results["f64acc"][0]) * 1e-3)
                     / 1e9, "f64acc_ms_per_step": f64_ms,
                     "kahan_ms_per_step": step_ms,
                     "kahan_direct_ms_per_step": (statistics.mean(results["kahan_direct"][0])
                                                  if "kahan_direct" in results else None),
                     "lognormal_65536_per_precision": variants},
        "adjoint": adj,
        "batched": batched,
        "batched_sharded": batched_sharded,
        "sharded": sharded,
        "paper_workload": paper,
    }
    if ws == 1 and not args.skip_cpu:
        line["cpu_baseline"], line["accuracy"] = cpu_baseline(args.cpu_seconds, first,
                                                              first65536)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_profile_case(args):
    """A few nb_forces calls at --profile N (--precision, default positions
    and pairs): the small and full-size cases of the ncu captures under
    profiles/."""
    import torch

    import paper_2605_02744_gb300 as pkg
    from paper_2605_02744_gb300 import api, ics
    pkg.build()
    n = int(args.profile)
    s = ics.plummer(n, seed=0)
    pos = torch.tensor(s.pos, device="cuda")
    mass = torch.tensor(s.mass, device="cuda")
    for _ in range(args.warmup + args.steps):
        api.forces(pos, mass, EPS_MAIN, precision=args.precision)
    torch.cuda.synchronize()
    return 0


def run_profile_adjoint(args):
    """--profile-adjoint: the adjoint workload once (16384 particles, 200
    KDK steps of 1e-3, eps 5e-3, F64ACC): the forward steps and one
    time-reversed gradient (the case its ncu captures used)."""
    import torch

    import paper_2605_02744_gb300 as pkg
    from paper_2605_02744_gb300 import adjoint, ics
    pkg.build()
    s = ics.plummer(16384, seed=0)
    target = ics.perturb_positions(s.pos, 1e-3, seed=2)
    adjoint.time_forward_backward(s, target, eps=5e-3, dt=1e-3, nsteps=200, segment=20,
                                  precision="f64acc", modes=("reverse",), reps=1)
    torch.cuda.synchronize()
    return 0


def run_profile_batched(args):
    """--profile-batched B: the batched path on the first B clusters of the
    512-cluster workload (F64ACC, dt = 1e-3): one system object, then
    warmup + steps calls of 100 KDK steps each (the case its ncu captures
    used)."""
    import numpy as np
    import torch

    import paper_2605_02744_gb300 as pkg
    from paper_2605_02744_gb300 import api, ics
    pkg.build()
    sizes = ics.batched_sizes()[: args.profile_batched]
    s = ics.batched_plummer(b=len(sizes), seed=1, sizes=sizes)
    g = api.System(s.pos, s.vel, s.mass, np.full(len(sizes), 0.01), offsets=s.offsets,
                   precision="f64acc")
    for _ in range(args.warmup + args.steps):
        g.step(1e-3, 100)
    torch.cuda.synchronize()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-adjoint", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-extra", action="store_true",
                    help="skip the batched and per-precision side measurements")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--profile", type=int, default=0,
                    help="run only nb_forces on a Plummer sphere of this size (for ncu)")
    ap.add_argument("--precision", default="kahan")
    ap.add_argument("--profile-batched", type=int, default=0,
                    help="run only the batched kernel on this many clusters (for ncu)")
    ap.add_argument("--profile-adjoint", action="store_true",
                    help="run only the adjoint workload's forward and one gradient (for ncu)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile_case(args)
    if args.profile_batched:
        return run_profile_batched(args)
    if args.profile_adjoint:
        return run_profile_adjoint(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
