"""Tensor-level conveniences over the C ABI.

These only allocate outputs and the workspace with torch, marshal arguments
and call the binding; the arithmetic is the library's.
"""
from __future__ import annotations

import torch

from . import binding as B


def _dev_f64(x, device):
    return torch.as_tensor(x, dtype=torch.float64).to(device).contiguous()


def _resolve_tune(tune, kind, precision, n, autotune):
    """tune="auto": the cached choice for this device and size, tuned on a miss."""
    if tune != "auto":
        return tune
    from . import tune as T
    hit = T.lookup(kind, precision, n)
    return hit if hit is not None else autotune()


def forces(pos, mass, eps: float, precision="f64acc", G: float = 1.0, with_pot: bool = True,
           tune=None, ws=None, stream=None, positions="default", pairs="default"):
    """(acc, pot) for one system; pos [N,3], mass [N] CUDA float64 tensors.

    tune: None (built-in shapes), an nb_tune dict, or "auto" (autotuner cache).
    positions / pairs: nb_positions / nb_pairs names ("default", "split",
    "single", "adaptive" / "default", "direct", "symmetric").
    """
    if tune == "auto":
        from . import tune as T
        tune = _resolve_tune(tune, "force", precision, mass.shape[0],
                             lambda: T.autotune_forces(pos, mass, eps, precision))
    opts = B.make_opts(precision, G, stream, tune=tune, positions=positions, pairs=pairs)
    n = mass.shape[0]
    acc = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
    pot = torch.empty(n, dtype=torch.float64, device=pos.device) if with_pot else None
    if ws is None:
        ws = B.workspace(n, 1, opts, pos.device)
    B.nb_forces(pos, mass, eps, acc, pot, ws, opts)
    return acc, pot


def forces_host(pos, mass, eps: float, precision="f64acc", G: float = 1.0, tune=None, ws=None,
                device="cuda"):
    """End-to-end call from host arrays: pinned H2D copies, nb_forces, D2H copies.

    pos, mass: numpy or CPU tensors (float64).  Returns CPU tensors (acc, pot).
    """
    hp = torch.as_tensor(pos, dtype=torch.float64).contiguous().pin_memory()
    hm = torch.as_tensor(mass, dtype=torch.float64).contiguous().pin_memory()
    dp = hp.to(device, non_blocking=True)
    dm = hm.to(device, non_blocking=True)
    acc, pot = forces(dp, dm, eps, precision, G, True, tune, ws)
    ha = torch.empty(acc.shape, dtype=torch.float64, pin_memory=True)
    hpot = torch.empty(pot.shape, dtype=torch.float64, pin_memory=True)
    ha.copy_(acc, non_blocking=True)
    hpot.copy_(pot, non_blocking=True)
    torch.cuda.current_stream().synchronize()
    return ha, hpot


def forces_batched(pos, mass, offsets, eps, precision="f64acc", G: float = 1.0, ws=None,
                   stream=None, pairs="default"):
    """(acc, pot) for B independent clusters described by CSR offsets;
    pairs: "default"/"symmetric" (symmetric batched path) or "direct"."""
    opts = B.make_opts(precision, G, stream, pairs=pairs)
    n = mass.shape[0]
    nb = offsets.shape[0] - 1
    acc = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
    pot = torch.empty(n, dtype=torch.float64, device=pos.device)
    if ws is None:
        ws = B.workspace(n, nb, opts, pos.device)
    B.nb_forces_batched(pos, mass, offsets, eps, acc, pot, ws, opts)
    return acc, pot


class System:
    """Device-resident particle state advanced with nb_step.

    Single system (offsets None, scalar eps) or a batch of independent
    clusters (offsets int64 [B+1], eps float64 [B]).
    """

    def __init__(self, pos, vel, mass, eps, offsets=None, precision="f64acc", G: float = 1.0,
                 tune=None, device="cuda", stream=None, use_graph: bool = False,
                 positions="default", pairs="default"):
        self.device = torch.device(device)
        self.pos = _dev_f64(pos, self.device)
        self.vel = _dev_f64(vel, self.device)
        self.mass = _dev_f64(mass, self.device)
        n = self.mass.shape[0]
        if tune == "auto":
            from . import tune as T
            if offsets is None:
                tune = _resolve_tune(tune, "force", precision, n,
                                     lambda: T.autotune_forces(self.pos, self.mass, eps,
                                                               precision))
            else:
                kind = "batched-" + T.batched_pairs(precision, pairs)
                tune = _resolve_tune(tune, kind, precision, n,
                                     lambda: T.autotune_batched(self.pos, self.vel, self.mass,
                                                                offsets, eps, 1e-3,
                                                                precision=precision,
                                                                pairs=pairs))
        self.acc = torch.zeros((n, 3), dtype=torch.float64, device=self.device)
        self.pot = torch.zeros(n, dtype=torch.float64, device=self.device)
        self.opts = B.make_opts(precision, G, stream, use_graph=use_graph, tune=tune,
                                positions=positions, pairs=pairs)
        if offsets is None:
            self.offsets = None
            self.eps_b = None
            self.eps = float(eps)
            nb = 1
        else:
            self.offsets = torch.as_tensor(offsets, dtype=torch.int64).to(self.device)
            nb = self.offsets.shape[0] - 1
            e = torch.as_tensor(eps, dtype=torch.float64)
            if e.dim() == 0:
                e = e.expand(nb)
            self.eps_b = e.contiguous().to(self.device)
            self.eps = 0.0
        self.ws = B.workspace(n, nb, self.opts, self.device)
        self.state = B.make_state(self.pos, self.vel, self.mass, self.acc, self.pot, self.eps,
                                  self.ws, self.offsets, self.eps_b)
        self._e = torch.zeros(3, dtype=torch.float64, device=self.device)

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])

    def step(self, dt: float, nsteps: int = 1):
        B.nb_step(self.state, dt, nsteps, self.opts)

    def forces(self):
        """Refresh acc/pot at the current positions."""
        self.state.acc_valid = 0
        B.nb_step(self.state, 0.0, 0, self.opts)

    def energy(self):
        """(K, W, E) as a device tensor of 3 doubles (pot must be current)."""
        B.nb_energy(self.state, self._e, self.opts)
        return self._e

    def poll(self) -> int:
        return B.nb_poll_status(self.ws, self.opts)
