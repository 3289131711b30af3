"""Shared helpers for the GPU parity tests (inputs from the seeded generator; expected
values from the FP64 oracle only)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def psnr(x, x_true, peak=255.0):
    mse = float(np.mean((np.asarray(x, np.float64) - x_true) ** 2))
    return 10.0 * np.log10(peak * peak / mse)


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.float32))).cuda()


def to_host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def f32(a):
    """The float32 rounding of an array, as float64 (what both sides are fed)."""
    return np.asarray(a, np.float32).astype(np.float64)
