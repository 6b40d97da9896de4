"""Pins of the oracle's force VJP and its discrete KDK adjoint.

The oracle's Jacobian blocks are derived by hand; here they are checked
against automatic differentiation (torch float64 on the CPU) of a dense
restatement of the forward map, against central finite differences of the
oracle's own forward map (dot-product test), and the trajectory adjoint is
checked against finite differences of the final-position loss.
"""
import numpy as np
import pytest
import torch

from paper_2605_02744_gb300 import ics


def _dense_forces_torch(x, m, eps, G=1.0):
    d = x[None, :, :] - x[:, None, :]  # d[i, j] = x_j - x_i
    s2 = (d * d).sum(-1) + eps * eps
    n = x.shape[0]
    off = 1.0 - torch.eye(n, dtype=x.dtype)
    w = m[None, :] * off
    a = G * (w[:, :, None] * d / s2[:, :, None] ** 1.5).sum(1)
    phi = -G * (w / s2.sqrt()).sum(1)
    return a, phi


@pytest.mark.parametrize("with_phibar", [False, True])
def test_vjp_matches_autograd(oracle_mod, with_phibar):
    n, eps, G = 64, 0.05, 1.7
    s = ics.plummer_lognormal(n, seed=3)
    rng = np.random.default_rng(4)
    abar = rng.normal(size=(n, 3))
    phibar = rng.normal(size=n) if with_phibar else None
    xb, mb = oracle_mod.forces_vjp(s.pos, s.mass, eps, abar, phibar, G=G)

    x = torch.tensor(s.pos, requires_grad=True)
    m = torch.tensor(s.mass, requires_grad=True)
    a, phi = _dense_forces_torch(x, m, eps, G)
    L = (a * torch.tensor(abar)).sum()
    if with_phibar:
        L = L + (phi * torch.tensor(phibar)).sum()
    gx, gm = torch.autograd.grad(L, (x, m))
    np.testing.assert_allclose(xb, gx.numpy(), rtol=1e-11, atol=1e-11 * np.abs(xb).max())
    np.testing.assert_allclose(mb, gm.numpy(), rtol=1e-11, atol=1e-11 * np.abs(mb).max())


def test_vjp_dot_product_with_finite_differences(oracle_mod):
    n, eps = 40, 0.02
    s = ics.plummer(n, seed=5)
    rng = np.random.default_rng(6)
    abar, phibar = rng.normal(size=(n, 3)), rng.normal(size=n)
    dx, dm = rng.normal(size=(n, 3)), rng.normal(size=n) * s.mass
    xb, mb = oracle_mod.forces_vjp(s.pos, s.mass, eps, abar, phibar)
    lhs = (xb * dx).sum() + (mb * dm).sum()
    h = 1e-5
    ap, pp = oracle_mod.forces(s.pos + h * dx, s.mass + h * dm, eps)
    am, pm = oracle_mod.forces(s.pos - h * dx, s.mass - h * dm, eps)
    rhs = ((ap - am) * abar).sum() / (2 * h) + ((pp - pm) * phibar).sum() / (2 * h)
    assert abs(lhs - rhs) <= 1e-7 * (abs(lhs) + 1e-30)


def _torch_kdk_loss(x, v, m, eps, h, nsteps, target):
    a, _ = _dense_forces_torch(x, m, eps)
    for _ in range(nsteps):
        v = v + 0.5 * h * a
        x = x + h * v
        a, _ = _dense_forces_torch(x, m, eps)
        v = v + 0.5 * h * a
    return ((x - target) ** 2).sum() / x.shape[0]


def test_trajectory_adjoint_matches_autograd(oracle_mod):
    n, eps, h, steps = 16, 0.05, 1e-2, 12
    s = ics.plummer(n, seed=7)
    target = ics.perturb_positions(s.pos, 1e-2, seed=8)
    L, gx, gv, gm = oracle_mod.trajectory_loss_grad(s.pos, s.vel, s.mass, eps, h, steps,
                                                    target)
    x = torch.tensor(s.pos, requires_grad=True)
    v = torch.tensor(s.vel, requires_grad=True)
    m = torch.tensor(s.mass, requires_grad=True)
    Lt = _torch_kdk_loss(x, v, m, eps, h, steps, torch.tensor(target))
    tx, tv, tm = torch.autograd.grad(Lt, (x, v, m))
    assert abs(L - Lt.item()) <= 1e-13 * abs(L)
    for ours, ref in ((gx, tx), (gv, tv), (gm, tm)):
        ref = ref.numpy()
        np.testing.assert_allclose(ours, ref, rtol=1e-9, atol=1e-10 * np.abs(ref).max())


def test_trajectory_adjoint_matches_finite_differences(oracle_mod):
    n, eps, h, steps = 24, 0.02, 5e-3, 20
    s = ics.plummer_lognormal(n, seed=9)
    target = ics.perturb_positions(s.pos, 1e-3, seed=2)
    _, gx, gv, gm = oracle_mod.trajectory_loss_grad(s.pos, s.vel, s.mass, eps, h, steps,
                                                    target)
    grad = np.concatenate([gx.ravel(), gv.ravel(), gm])
    coords = ics.random_coordinates(n, k=12, seed=3)
    base = [s.pos, s.vel, s.mass]
    for c in coords:
        pert = []
        for sign in (1.0, -1.0):
            p, v, m = (b.copy() for b in base)
            if c < 3 * n:
                step = 1e-6
                p.reshape(-1)[c] += sign * step
            elif c < 6 * n:
                step = 1e-6
                v.reshape(-1)[c - 3 * n] += sign * step
            else:
                step = 1e-6 * s.mass[c - 6 * n]
                m[c - 6 * n] += sign * step
            pert.append(oracle_mod.final_loss(p, v, m, eps, h, steps, target))
        fd = (pert[0] - pert[1]) / (2 * step)
        assert abs(fd - grad[c]) <= 1e-6 * max(abs(grad[c]), 1e-3 * np.abs(grad).max())
