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


# Bars of the FP32 path against the FP64 oracle from the same float32 inputs.
SOLVE_REL_L2 = 1e-3      # relative L2 of a whole solve
SOLVE_PSNR_DB = 0.01     # |PSNR difference| of a whole solve
SOLVE_MAX_ABS = 0.5      # every pixel of a solve within half a grey level of [0, 255]
STEP_REL_L2 = 1e-5       # one FP step or one linear solve
STEP_MAX_ABS = 2e-3      # every pixel of one step (the NLM bar: ex2.approx + FP32 sums)


def solve_errors(x, x_ref, x_true):
    x = np.asarray(x, np.float64)
    x_ref = np.asarray(x_ref, np.float64)
    return {"rel_l2": rel_l2(x, x_ref), "psnr_db": abs(psnr(x, x_true) - psnr(x_ref, x_true)),
            "max_abs": float(np.abs(x - x_ref).max())}


def assert_solve_close(x, x_ref, x_true, label="", rel=SOLVE_REL_L2, db=SOLVE_PSNR_DB,
                       max_abs=SOLVE_MAX_ABS):
    """A GPU solve against the oracle's: relative L2, PSNR and element-wise bars."""
    e = solve_errors(x, x_ref, x_true)
    msg = (f"{label}: rel L2 {e['rel_l2']:.3e} (bar {rel:g}), PSNR diff {e['psnr_db']:.5f} dB "
           f"(bar {db:g}), max abs {e['max_abs']:.4e} (bar {max_abs:g})")
    print(msg)
    assert e["rel_l2"] <= rel and e["psnr_db"] <= db and e["max_abs"] <= max_abs, msg
    return e


def assert_step_close(x, ref, label="", rel=STEP_REL_L2, max_abs=STEP_MAX_ABS):
    """One FP step (or linear solve, or extrapolation) against the oracle: relative L2 and
    element-wise bars."""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    r = rel_l2(x, ref)
    m = float(np.abs(x - ref).max())
    msg = f"{label}: rel L2 {r:.3e} (bar {rel:g}), max abs {m:.4e} (bar {max_abs:g})"
    print(msg)
    assert r <= rel and m <= max_abs, msg
    return r, m


# How far a solve's result may move under per-step errors of the FP32 path's size: the
# oracle's own solve with every FP step's output rounded to 20 or 19 significant bits
# (relative 2^-21 or 2^-20: the measured per-step error of the GPU path in L2 and at its
# worst pixels) against the exact FP64 solve. Where the extrapolation weights are large
# (sum |gamma|, Eq. (21)) this distance exceeds the FP32 bars; the GPU must then stay
# within ENVELOPE_FACTOR times the larger of the two.
ENVELOPE_FACTOR = 3.0


def solve_bars(sensitivity=None, factor=ENVELOPE_FACTOR):
    """(rel, db, max_abs) bars of a solve: the FP32 bars, or factor x the method's measured
    sensitivity where that is larger."""
    if sensitivity is None:
        return SOLVE_REL_L2, SOLVE_PSNR_DB, SOLVE_MAX_ABS
    return (max(SOLVE_REL_L2, factor * sensitivity["rel_l2"]),
            max(SOLVE_PSNR_DB, factor * sensitivity["psnr_db"]),
            max(SOLVE_MAX_ABS, factor * sensitivity["max_abs"]))


def oracle_sensitivity(make_map, x0, x_ref, x_true, method, m, kappa, calls, bits=(20, 19),
                       **kw):
    """Largest distance, over the given roundings, of the oracle's solve with every FP
    output rounded to that many significant bits from its exact solve x_ref (see
    ENVELOPE_FACTOR)."""
    import sys
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    if here not in sys.path:
        sys.path.insert(0, here)
    from make_full_size_oracle import Rounded
    from oracle import red as ored
    worst = None
    for b in bits:
        xp, _ = ored.solve(Rounded(make_map(), b), x0, method, m=m, kappa=kappa,
                           max_calls=calls, **kw)
        e = solve_errors(xp, x_ref, x_true)
        worst = e if worst is None else {k: max(worst[k], e[k]) for k in e}
    return worst
