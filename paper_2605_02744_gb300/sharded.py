"""One system's leapfrog split over the ranks of a process group.

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
