"""Work split over the ranks of a process group: one system's leapfrog by
rows (ShardedSystem), or a batch of independent clusters by cluster
(ShardedBatch).

The particles are cut into contiguous ranges, one per rank -- the data
decomposition of the paper's first multi-device strategy (Sec. 3.2,
approach 1: every device computes the forces of its own particles against
all of them).  Rank r owns rows [r c, min((r + 1) c, N)) with c = ceil(N / P).
A kick-drift-kick step on every rank:

1. ``nb_kick_drift(h/2, h)`` on its own rows (opening kick and drift);
2. all-gather of the positions -- the only exchange: P chunks of c rows
   (the last rank's chunk padded), so the gathered buffer's first N rows are
   the system in particle order;
3. ``nb_forces_range`` for its own rows against all N at the new positions;
4. ``nb_kick_drift(h/2, 0)`` (closing kick).

Energies are summed over ranks with one all-reduce.  The forces of a rank do
not depend on how the others are cut, so the result equals the single-GPU
direct-kernel step up to the summation order inside the kernel.

The arithmetic runs in the library's CUDA kernels (``LibraryOps``); torch
provides the device buffers and the collective.  The ops object is a
parameter so that the partitioning, gather order and reassembly can be
exercised by tests with a stand-in.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as B


def partition(n: int, world: int, rank: int):
    """(i0, i1, c): rank's rows [i0, i1) and the chunk size c = ceil(n / world)
    of the gather (the last ranks may own fewer than c rows, even none)."""
    if n < 1 or world < 1 or not 0 <= rank < world:
        raise ValueError("need n >= 1, world >= 1, 0 <= rank < world")
    c = math.ceil(n / world)
    i0 = min(rank * c, n)
    i1 = min(i0 + c, n)
    return i0, i1, c


def _dist_state(group):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(group), dist.get_rank(group)
    return 1, 0


class LibraryOps:
    """The GPU implementation: library kernels through the C ABI."""

    def __init__(self, n, precision, device, stream=None, positions="default"):
        self.opts = B.make_opts(precision, stream=stream, positions=positions, pairs="direct")
        self.ws = B.workspace(n, 1, self.opts, device)

    def forces_range(self, pos_all, mass_all, eps, i0, i1, acc, pot):
        B.nb_forces_range(pos_all, mass_all, i0, i1, eps, acc, pot, self.ws, self.opts)

    def kick_drift(self, pos, vel, acc, kick, drift):
        B.nb_kick_drift(pos, vel, acc, kick, drift, self.opts)

    def energy_rows(self, pos, vel, acc, mass, pot):
        """(K, W) of the rows, summed on the device by the library."""
        out = torch.empty(3, dtype=torch.float64, device=vel.device)
        st = B.make_state(pos, vel, mass, acc, pot, 1.0, self.ws)
        B.nb_energy(st, out, self.opts)
        return out[:2]

    def vjp_range(self, pos_all, mass_all, eps, i0, i1, coef, abar_all, pos_bar, mass_bar):
        """pos_bar / mass_bar (the rows) += coef x the rows' VJP of the
        cotangents abar_all of all N particles."""
        B.nb_forces_vjp_range(pos_all, mass_all, i0, i1, eps, coef, abar_all, None, pos_bar,
                              mass_bar, self.ws, self.opts)

    def kick(self, vel, acc, kick):
        """vel += kick acc (the library's kick with no drift)."""
        B.nb_kick_drift(vel, vel, acc, kick, 0.0, self.opts)

    def poll(self):
        return B.nb_poll_status(self.ws, self.opts)


class ShardedSystem:
    """KDK leapfrog of N particles whose rows are split over the group's ranks.

    pos, vel, mass: the whole system (array-likes of shape [N, 3], [N, 3],
    [N]), the same on every rank.  After construction and after every
    ``step`` each rank's ``acc`` / ``pot`` hold its rows at its current
    positions.
    """

    def __init__(self, pos, vel, mass, eps: float, precision="f64acc", group=None,
                 device=None, ops=None):
        self.group = group
        self.world, self.rank = _dist_state(group)
        mass_t = torch.as_tensor(mass, dtype=torch.float64)
        n = mass_t.shape[0]
        self.n = n
        self.eps = float(eps)
        self.i0, self.i1, self.c = partition(n, self.world, self.rank)
        self.rows = self.i1 - self.i0
        dev = torch.device(device) if device is not None else (
            torch.device("cuda", torch.cuda.current_device()) if ops is None else
            torch.device("cpu"))
        self.device = dev
        self.ops = ops if ops is not None else LibraryOps(n, precision, dev)
        f64 = dict(dtype=torch.float64, device=dev)
        pos_t = torch.as_tensor(pos, dtype=torch.float64)
        vel_t = torch.as_tensor(vel, dtype=torch.float64)
        self.mass = mass_t.to(dev).contiguous()
        # the gather buffer: world chunks of c rows; rows >= n are padding
        self.gathered = torch.zeros((self.world * self.c, 3), **f64)
        self.pos_all = self.gathered[:n]
        self.chunk = torch.zeros((self.c, 3), **f64)  # this rank's rows, padded
        self.chunk[:self.rows] = pos_t[self.i0:self.i1].to(dev)
        self.pos = self.chunk[:self.rows]
        self.vel = vel_t[self.i0:self.i1].to(dev).contiguous()
        self.acc = torch.zeros((self.rows, 3), **f64)
        self.pot = torch.zeros(self.rows, **f64)
        self.step_count = 0
        self._gather()
        self._forces()

    def _gather(self):
        if self.world == 1:
            self.gathered[:self.c].copy_(self.chunk)
            return
        import torch.distributed as dist
        if dist.get_backend(self.group) == "nccl":
            dist.all_gather_into_tensor(self.gathered, self.chunk, group=self.group)
        else:
            parts = list(self.gathered.view(self.world, self.c, 3).unbind(0))
            dist.all_gather(parts, self.chunk, group=self.group)

    def gather_rows(self, rows):
        """All N rows of a per-rank [rows, 3] tensor, in particle order (one
        all-gather of c-row chunks)."""
        chunk = torch.zeros((self.c, 3), dtype=rows.dtype, device=rows.device)
        chunk[:self.rows] = rows
        if self.world == 1:
            return chunk[:self.n].clone()
        out = torch.empty((self.world * self.c, 3), dtype=rows.dtype, device=rows.device)
        import torch.distributed as dist
        if dist.get_backend(self.group) == "nccl":
            dist.all_gather_into_tensor(out, chunk, group=self.group)
        else:
            dist.all_gather(list(out.view(self.world, self.c, 3).unbind(0)), chunk,
                            group=self.group)
        return out[:self.n]

    def _forces(self):
        if self.rows > 0:
            self.ops.forces_range(self.pos_all, self.mass, self.eps, self.i0, self.i1, self.acc,
                                  self.pot)

    def step(self, dt: float, nsteps: int = 1):
        for _ in range(int(nsteps)):
            if self.rows > 0:
                self.ops.kick_drift(self.pos, self.vel, self.acc, 0.5 * dt, dt)
            self._gather()
            self._forces()
            if self.rows > 0:
                self.ops.kick_drift(self.pos, self.vel, self.acc, 0.5 * dt, 0.0)
            self.step_count += 1

    def energy(self):
        """(K, W, E) of the whole system (sum over ranks of each rank's rows)."""
        if self.rows > 0:
            kw = self.ops.energy_rows(self.pos, self.vel, self.acc, self.mass[self.i0:self.i1],
                                      self.pot)
        else:
            kw = torch.zeros(2, dtype=torch.float64, device=self.device)
        kw = kw.clone()
        if self.world > 1:
            import torch.distributed as dist
            dist.all_reduce(kw, group=self.group)
        return torch.stack([kw[0], kw[1], kw[0] + kw[1]])

    def gather_state(self):
        """Positions, velocities, accelerations of all N particles (every rank)."""
        out = []
        for t in (self.pos, self.vel, self.acc):
            buf = torch.zeros((self.world * self.c, 3), dtype=torch.float64, device=self.device)
            chunk = torch.zeros((self.c, 3), dtype=torch.float64, device=self.device)
            chunk[:self.rows] = t
            if self.world == 1:
                buf[:self.c].copy_(chunk)
            else:
                import torch.distributed as dist
                parts = list(buf.view(self.world, self.c, 3).unbind(0))
                dist.all_gather(parts, chunk, group=self.group)
            out.append(buf[:self.n])
        return tuple(out)


def partition_clusters(sizes, world: int):
    """Cluster indices of each rank for a batch of independent systems.

    Each cluster costs N_c^2 pair terms per evaluation; clusters go, largest
    first (ties: lower index), to the rank with the least cost so far (ties:
    lower rank).  Each rank's list is in ascending cluster order.  Clusters
    share no particles, so nothing crosses ranks while they are stepped.
    """
    sizes = [int(x) for x in sizes]
    if world < 1 or any(n < 0 for n in sizes):
        raise ValueError("need world >= 1 and sizes >= 0")
    load = [0] * world
    out = [[] for _ in range(world)]
    for c in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(c)
        load[r] += sizes[c] ** 2
    return [sorted(x) for x in out]


class LibraryBatchOps:
    """The GPU implementation for a rank's clusters: the library's batched
    path (one api.System over them)."""

    def __init__(self, pos, vel, mass, offsets, eps, precision, device, **system_kw):
        from .api import System
        self.sys = System(pos, vel, mass, eps, offsets=offsets, precision=precision,
                          device=device, **system_kw)

    def step(self, dt, nsteps):
        self.sys.step(dt, nsteps)

    def energy_kw(self):
        return self.sys.energy()[:2]

    def state(self):
        return self.sys.pos, self.sys.vel, self.sys.acc

    def poll(self):
        return self.sys.poll()


class ShardedBatch:
    """A batch of independent clusters split over the ranks by cluster.

    pos, vel, mass: all clusters' particles (array-likes [N, 3], [N, 3], [N]),
    offsets: CSR cluster boundaries [B + 1], eps: one softening length per
    cluster (or a scalar) -- the same on every rank.  Rank r advances the
    clusters partition_clusters(sizes, world)[r] with the batched path; the
    steps exchange nothing.  A cluster's arithmetic does not depend on which
    other clusters share its launch, so each cluster's trajectory is the one
    a single-GPU run of the whole batch gives.  world / rank default to the
    process group's (or 1 / 0 without one); passing them runs one rank's
    share in this process.
    """

    def __init__(self, pos, vel, mass, offsets, eps, precision="f64acc", group=None, device=None,
                 ops=None, world=None, rank=None, **system_kw):
        self.group = group
        if world is None:
            self.world, self.rank = _dist_state(group)
            self.collective = self.world > 1
        else:
            self.world, self.rank = int(world), int(rank)
            self.collective = False
        offsets = np.asarray(offsets, dtype=np.int64)
        sizes = np.diff(offsets)
        b = sizes.shape[0]
        eps_all = np.broadcast_to(np.asarray(eps, dtype=np.float64), (b,))
        self.n = int(offsets[-1])
        self.clusters = partition_clusters(sizes, self.world)[self.rank]
        self.rows = (np.concatenate([np.arange(offsets[c], offsets[c + 1]) for c in self.clusters])
                     if self.clusters else np.zeros(0, dtype=np.int64))
        self.local_offsets = np.r_[0, np.cumsum(sizes[self.clusters])].astype(np.int64)
        dev = torch.device(device) if device is not None else (
            torch.device("cuda", torch.cuda.current_device()) if ops is None else
            torch.device("cpu"))
        self.device = dev
        if ops is None and self.clusters:
            pos, vel, mass = (np.asarray(a, dtype=np.float64) for a in (pos, vel, mass))
            ops = LibraryBatchOps(pos[self.rows], vel[self.rows], mass[self.rows],
                                  self.local_offsets, eps_all[self.clusters].copy(), precision,
                                  dev, **system_kw)
        elif ops is not None:
            ops.bind(np.asarray(pos, dtype=np.float64)[self.rows],
                     np.asarray(vel, dtype=np.float64)[self.rows],
                     np.asarray(mass, dtype=np.float64)[self.rows], self.local_offsets,
                     eps_all[self.clusters].copy())
        self.ops = ops if self.clusters else None

    def step(self, dt: float, nsteps: int = 1):
        if self.ops is not None:
            self.ops.step(dt, nsteps)

    def energy(self):
        """(K, W, E) of the whole batch (one all-reduce over the ranks)."""
        if self.ops is not None:
            kw = self.ops.energy_kw().clone()
        else:
            kw = torch.zeros(2, dtype=torch.float64, device=self.device)
        if self.collective:
            import torch.distributed as dist
            dist.all_reduce(kw, group=self.group)
        return torch.stack([kw[0], kw[1], kw[0] + kw[1]])

    def local_state(self):
        """(rows, pos, vel, acc): this rank's particle indices and state."""
        if self.ops is None:
            z = torch.zeros((0, 3), dtype=torch.float64, device=self.device)
            return self.rows, z, z, z
        return (self.rows, *self.ops.state())

    def gather_state(self):
        """Positions, velocities, accelerations of all N particles as host
        arrays, on every rank (one all-gather of the ranks' rows)."""
        rows, p, v, a = self.local_state()
        mine = (rows, p.cpu().numpy(), v.cpu().numpy(), a.cpu().numpy())
        if self.collective:
            import torch.distributed as dist
            parts = [None] * self.world
            dist.all_gather_object(parts, mine, group=self.group)
        else:
            parts = [mine]
        out = [np.zeros((self.n, 3)) for _ in range(3)]
        for rows, *arrs in parts:
            for o, x in zip(out, arrs):
                o[rows] = x
        return tuple(out)


def sharded_loss_and_grads(pos, vel, mass, eps: float, h: float, nsteps: int, target,
                           precision="f64acc", group=None, device=None, ops=None):
    """L = (1/N) sum_i |x_i(T) - x*_i|^2 after nsteps KDK steps of one system
    whose rows are split over the ranks (ShardedSystem), and the gradients of
    L with respect to the rank's rows of the initial positions, velocities
    and masses: the discrete adjoint of each step, unmerged.

    Forward: the sharded steps, keeping the gathered positions of every step
    ((nsteps + 1) N 24 bytes per rank).  Reverse, per step (with u the rows'
    velocity cotangent): an all-gather of u, the rows' VJP at x_(k+1) with
    coefficient h/2, u += h xbar, a second all-gather, the rows' VJP at x_k
    with coefficient h/2: two all-gathers of cotangents per step on top of
    the forward pass's one of positions.

    Returns (L, xbar, vbar, mbar, (i0, i1)) with the rows' gradients.
    """
    g = ShardedSystem(pos, vel, mass, eps, precision=precision, group=group, device=device,
                      ops=ops)
    xs = [g.pos_all.clone()]
    for _ in range(int(nsteps)):
        g.step(h, 1)
        xs.append(g.pos_all.clone())
    tgt = torch.as_tensor(target, dtype=torch.float64)[g.i0:g.i1].to(g.device)
    d = xs[-1][g.i0:g.i1] - tgt
    part = (d * d).sum().reshape(1)
    if g.world > 1:
        import torch.distributed as dist
        dist.all_reduce(part, group=group)
    L = float(part.item()) / g.n
    f64 = dict(dtype=torch.float64, device=g.device)
    xbar = (2.0 / g.n) * d
    vbar = torch.zeros((g.rows, 3), **f64)
    mbar = torch.zeros(g.rows, **f64)
    for k in range(int(nsteps) - 1, -1, -1):
        if g.rows > 0:
            g.ops.vjp_range(xs[k + 1], g.mass, g.eps, g.i0, g.i1, 0.5 * h,
                            g.gather_rows(vbar), xbar, mbar)
            g.ops.kick(vbar, xbar, h)
            g.ops.vjp_range(xs[k], g.mass, g.eps, g.i0, g.i1, 0.5 * h, g.gather_rows(vbar),
                            xbar, mbar)
        else:  # still take part in the collectives
            g.gather_rows(vbar)
            g.gather_rows(vbar)
    return L, xbar, vbar, mbar, (g.i0, g.i1)
