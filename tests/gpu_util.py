"""Shared helpers of the GPU parity tests (error metrics, device transfer)."""
import numpy as np
import torch


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_vec_err(a, ref):
    """Per-particle |a - ref| / |ref| (vector norm); zero rows compare absolutely."""
    num = np.linalg.norm(a - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def rel_err(p, ref):
    den = np.abs(ref)
    return np.where(den > 0, np.abs(p - ref) / np.where(den > 0, den, 1.0), np.abs(p - ref))


# Gates (relative, per particle, max over particles): FP32 pairs with Kahan or
# FP64 accumulation 1e-5; FP64 pairs 1e-12; all-FP32 accumulation is only
# reported at large N and gated loosely at small N.
TOL = {"kahan": 1e-5, "f64acc": 1e-5, "fp64": 1e-12, "fp32": 1e-4}
