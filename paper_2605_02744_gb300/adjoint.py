"""Gradients of a final-state loss through kick-drift-kick leapfrog.

``simulate(x0, v0, m, eps, dt, nsteps, segment)`` advances the system with
nb_step and is differentiable with respect to x0, v0 and m.  The backward
pass is the discrete adjoint of KDK built from the library's force VJP:
walking back from the final cotangents (xbar, vbar), every position state
x_k receives one VJP with cotangent c = coef * vbar after the drift adjoint
vbar += dt * xbar, where coef = dt/2 at x_K and x_0 and dt in between (the
two half-kicks that meet at x_k merged into one call; nb_step_vjp).

Memory is bounded by checkpoints: (x, v) is stored every ``segment`` steps.
Two ways to get the positions between checkpoints back:

* ``mode="recompute"`` re-runs the forward from each checkpoint, storing the
  segment's positions, then sweeps it backwards (one force + one VJP per
  step).
* ``mode="reverse"`` runs the leapfrog map backwards from the final state
  (it is time-reversible): nb_step_vjp_reverse evaluates a(x_k) and the VJP
  at x_k in one kernel and rewinds x_{k-1} = x_k - dt v_{k-1/2}; the state is
  re-anchored to the stored (x, v) at every checkpoint.

Torch only holds tensors and records the autograd graph; every force, VJP
and state update runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import binding as B


def _f64(x, device):
    return torch.as_tensor(x, dtype=torch.float64).to(device).contiguous()


class _Ctx:
    """Device buffers of one simulation (state, workspace, options)."""

    def __init__(self, x0, v0, m, eps, precision, G, stream, tune):
        dev = x0.device
        n = m.shape[0]
        self.n = n
        self.eps = float(eps)
        self.opts = B.make_opts(precision, G, stream, tune=tune)
        self.ws = B.workspace(n, 1, self.opts, dev)
        self.pos = x0.detach().clone().contiguous()
        self.vel = v0.detach().clone().contiguous()
        self.mass = m.detach().contiguous()
        self.acc = torch.zeros((n, 3), dtype=torch.float64, device=dev)
        self.state = B.make_state(self.pos, self.vel, self.mass, self.acc, None, self.eps,
                                  self.ws)

    def reset(self, x, v, a=None):
        self.pos.copy_(x)
        self.vel.copy_(v)
        if a is not None:
            self.acc.copy_(a)
        self.state.acc_valid = 0 if a is None else 1

    def step(self, dt, n):
        B.nb_step(self.state, dt, n, self.opts)


class _Leapfrog(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, m, eps, dt, nsteps, segment, precision, G, mode, tune):
        sim = _Ctx(x0, v0, m, eps, precision, G, None, tune)
        ckpts = []
        done = 0
        while done < nsteps:
            a = sim.acc.clone() if sim.state.acc_valid else None
            ckpts.append((done, sim.pos.clone(), sim.vel.clone(), a))
            k = min(segment, nsteps - done)
            sim.step(dt, k)
            done += k
        if nsteps == 0:
            sim.step(dt, 0)
        ctx.sim = sim
        ctx.ckpts = ckpts
        ctx.args = (float(dt), int(nsteps), int(segment), mode)
        ctx.save_for_backward(m)
        return sim.pos.clone(), sim.vel.clone()

    @staticmethod
    def backward(ctx, gx, gv):
        sim = ctx.sim
        dt, nsteps, segment, mode = ctx.args
        n = sim.n
        dev = sim.pos.device
        xbar = (gx if gx is not None else torch.zeros((n, 3), dtype=torch.float64,
                                                      device=dev)).contiguous().clone()
        vbar = (gv if gv is not None else torch.zeros((n, 3), dtype=torch.float64,
                                                      device=dev)).contiguous().clone()
        mbar = torch.zeros(n, dtype=torch.float64, device=dev)
        if nsteps == 0:
            return xbar, vbar, mbar, *([None] * 8)
        o = sim.opts
        if mode == "recompute":
            xK = sim.pos.clone()
            B.nb_step_vjp(xK, sim.mass, sim.eps, 0.0, 0.5 * dt, xbar, vbar, mbar, sim.ws, o)
            seg_pos = None
            for (c, xc, vc, ac) in reversed(ctx.ckpts):
                length = min(segment, nsteps - c)
                if seg_pos is None or seg_pos.shape[0] < length:
                    seg_pos = torch.empty((length, n, 3), dtype=torch.float64, device=dev)
                sim.reset(xc, vc, ac)
                seg_pos[0].copy_(xc)
                for k in range(1, length):
                    sim.step(dt, 1)
                    seg_pos[k].copy_(sim.pos)
                for k in range(length - 1, -1, -1):
                    coef = 0.5 * dt if c + k == 0 else dt
                    B.nb_step_vjp(seg_pos[k], sim.mass, sim.eps, dt, coef, xbar, vbar, mbar,
                                  sim.ws, o)
        elif mode == "reverse":
            # at x_K the state is (x_K, v_K): the first call's rewind kick is
            # dt/2 (v_K - dt/2 a_K = v_{K-1/2}); later ones carry v_{k+1/2}
            pos = sim.pos.clone()
            vhalf = sim.vel.clone()
            acc = torch.empty_like(pos)
            anchors = {c: (xc, vc) for (c, xc, vc, _) in ctx.ckpts}
            for k in range(nsteps, -1, -1):
                drift, coef = (0.0, 0.5 * dt) if k == nsteps else (dt, dt)
                if k == 0:
                    coef = 0.5 * dt
                rk, rd = (dt, dt) if k > 0 else (0.0, 0.0)
                if k == nsteps:
                    rk = 0.5 * dt
                if k in anchors and k != nsteps:
                    pos.copy_(anchors[k][0])
                    vhalf.copy_(anchors[k][1])
                    rk = 0.5 * dt if k > 0 else 0.0
                B.nb_step_vjp_reverse(pos, vhalf, acc, sim.mass, sim.eps, rk, rd, drift, coef,
                                      xbar, vbar, mbar, sim.ws, o)
        else:
            raise ValueError(f"unknown adjoint mode {mode!r}")
        return xbar, vbar, mbar, *([None] * 8)


def simulate(x0, v0, m, eps: float, dt: float, nsteps: int, segment: int = 20,
             precision="f64acc", G: float = 1.0, mode: str = "reverse", tune=None):
    """Final (x, v) after nsteps KDK steps; differentiable w.r.t. x0, v0, m."""
    if segment < 1:
        raise ValueError("segment must be >= 1")
    return _Leapfrog.apply(x0, v0, m, eps, dt, nsteps, segment, precision, G, mode, tune)


def loss_and_grads(pos, vel, mass, eps, dt, nsteps, target, segment=20, precision="f64acc",
                   mode="reverse", device="cuda"):
    """L = (1/N) sum |x(T) - target|^2 and its gradients w.r.t. (x0, v0, m)."""
    x0 = _f64(pos, device).requires_grad_(True)
    v0 = _f64(vel, device).requires_grad_(True)
    m = _f64(mass, device).requires_grad_(True)
    tgt = _f64(target, device)
    xT, _ = simulate(x0, v0, m, eps, dt, nsteps, segment, precision, mode=mode)
    L = ((xT - tgt) ** 2).sum() / xT.shape[0]
    gx, gv, gm = torch.autograd.grad(L, (x0, v0, m))
    return L.detach(), gx, gv, gm


def time_forward_backward(s, target, eps=5e-3, dt=1e-3, nsteps=200, segment=20,
                          precision="f64acc", modes=("reverse", "recompute"), reps=2):
    """CUDA-event times of the forward run and of the gradient, per mode."""
    dev = torch.device("cuda")
    out = {"N": int(s.n), "nsteps": nsteps, "segment": segment, "precision": precision}
    x0 = _f64(s.pos, dev)
    v0 = _f64(s.vel, dev)
    m = _f64(s.mass, dev)
    tgt = _f64(target, dev)
    sim = _Ctx(x0, v0, m, eps, precision, 1.0, None, None)

    def fwd():
        sim.reset(x0, v0)
        sim.step(dt, nsteps)

    ev = lambda: torch.cuda.Event(enable_timing=True)
    fwd()
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0, e1 = ev(), ev()
        e0.record()
        fwd()
        e1.record()
        e1.synchronize()
        best = min(best or 1e30, e0.elapsed_time(e1))
    out["forward_ms"] = best
    grads = {}
    for mode in modes:
        xs = x0.clone().requires_grad_(True)
        vs = v0.clone().requires_grad_(True)
        ms = m.clone().requires_grad_(True)
        tb = None
        for _ in range(reps):
            xT, _ = simulate(xs, vs, ms, eps, dt, nsteps, segment, precision, mode=mode)
            L = ((xT - tgt) ** 2).sum() / xT.shape[0]
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record()
            g = torch.autograd.grad(L, (xs, vs, ms))
            e1.record()
            e1.synchronize()
            tb = min(tb or 1e30, e0.elapsed_time(e1))
        grads[mode] = torch.cat([t.reshape(-1) for t in g])
        out[f"backward_ms_{mode}"] = tb
        out[f"ratio_{mode}"] = tb / best
    if "reverse" in grads and "recompute" in grads:
        a, b = grads["reverse"], grads["recompute"]
        out["reverse_vs_recompute_max_rel"] = float(((a - b).abs().max() / b.abs().max()).item())
    return out
