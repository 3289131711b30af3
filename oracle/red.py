"""RED objective and the cycling driver (Algorithm 3) in FP64.

Objective, Eq. (4):  E(x) = ||H x - y||^2 / (2 sigma^2) + (alpha / 2) x^T (x - f(x)).

Algorithm 3 (Sec. III-C), with these readings of what the paper leaves open:
  * a cycle runs m + kappa + 1 FP steps from its start vector x_0 and keeps
    x_m .. x_{m+kappa+1}; MPE / RRE / SVD-MPE (Algorithm 1 with the chosen step 2) gives
    x_(m,kappa), which becomes x_0 of the next cycle and costs no denoiser call;
  * termination is tested after every FP step: the relative change
    ||x_{i+1} - x_i||_2 / ||x_i||_2 < tol, or the budget of FP steps (denoiser calls)
    reached. The solve returns that FP iterate, so every extrapolated vector is followed
    by at least one FP step (the "additional iterations" remark of Sec. III-C);
  * on an extrapolation breakdown the next cycle starts from the last FP iterate.
  * with method "none" the driver is the plain FP iteration of Eq. (7);
  * cycling with frozen gamma (a remark of Sec. III-C; the paper leaves its details to the
    VE literature): after `freeze_after` cycles whose extrapolation succeeded, every later
    cycle runs m + kappa baseline steps and combines x_m .. x_{m+kappa} with the last
    computed gamma by Eq. (11), without the QR and the gamma solve (x_{m+kappa+1} is only
    needed to form U for the solve); before that, cycles are full;
  * the baseline map F may be any map of one denoiser call per step: the FP map of
    Eq. (7) (fp.FPOperator) or the steepest-descent step of SD-MPE (sd.SDOperator);
  * VE terminated by its own criterion, then baseline iterations (the "additional
    iterations ... after terminating the VE" remark of Sec. III-C): with ve_stop_tol > 0,
    the first FP step whose relative change falls below ve_stop_tol ends extrapolation;
    that cycle takes no extrapolation (the next start vector is the last FP iterate, as on
    a breakdown) and every later step is a plain FP step, until tol or the budget.
"""
from __future__ import annotations

import numpy as np

from . import operators as ops
from .ve import combine_direct, extrapolate


def objective(x: np.ndarray, fx: np.ndarray, y: np.ndarray, otf: np.ndarray, scale: int,
              sigma: float, alpha: float) -> float:
    r = ops.forward(x, otf, scale) - y
    return float(np.vdot(r, r)) / (2.0 * sigma ** 2) + 0.5 * alpha * float(np.vdot(x, x - fx))


def gradient(x: np.ndarray, fx: np.ndarray, y: np.ndarray, otf: np.ndarray, scale: int,
             sigma: float, alpha: float) -> np.ndarray:
    """Eq. (5): H^T (H x - y) / sigma^2 + alpha (x - f(x))."""
    r = ops.forward(x, otf, scale) - y
    return ops.adjoint(r, otf, scale, x.shape) / sigma ** 2 + alpha * (x - fx)


def psnr(x: np.ndarray, x_true: np.ndarray, peak: float = 255.0) -> float:
    mse = float(np.mean((np.asarray(x, np.float64) - x_true) ** 2))
    return 10.0 * np.log10(peak * peak / mse)


def rel_change(x_new: np.ndarray, x_old: np.ndarray) -> float:
    return float(np.linalg.norm((x_new - x_old).ravel()) / np.linalg.norm(x_old.ravel()))


def solve(F, x0: np.ndarray, method: str = "none", m: int = 0, kappa: int = 4,
          max_calls: int = 200, tol: float = 0.0, callback=None, freeze_after=None,
          ve_stop_tol: float = 0.0):
    """Algorithm 3 around the baseline map F. Returns (x, stats). `callback(calls, x)` is
    called after every baseline step (for convergence studies). `freeze_after`: None for
    full cycling, else the number of successful full cycles after which gamma is frozen.
    `ve_stop_tol`: extrapolation ends at the first FP step whose relative change is below
    it, and plain FP steps follow (0: never)."""
    if ve_stop_tol > 0.0 and freeze_after is not None:
        raise ValueError("ve_stop_tol and freeze_after do not combine")
    x = np.asarray(x0, dtype=np.float64).copy()
    calls = 0
    stats = {"fp_calls": 0, "ve_steps": 0, "ve_breakdowns": 0, "gammas": [],
             "sum_abs_gamma": [], "rel_change": None, "frozen_steps": 0, "ve_stopped_at": None}
    frozen = None
    while True:
        if stats["ve_stopped_at"] is not None:
            method = "none"

        # a frozen cycle needs x_m .. x_{m+kappa} only: x_{m+kappa+1} serves the gamma solve
        per_cycle = m + kappa + (1 if frozen is None else 0)
        stored = [x] if (method != "none" and m == 0) else []
        for i in range(1, per_cycle + 1):
            x_new = F(x)
            calls += 1
            rc = rel_change(x_new, x)
            x = x_new
            if callback is not None:
                callback(calls, x)
            if method != "none" and i >= m:
                stored.append(x)
            if method != "none" and stats["ve_stopped_at"] is None and rc < ve_stop_tol:
                stats["ve_stopped_at"] = calls
            if rc < tol or calls >= max_calls:
                stats.update(fp_calls=calls, rel_change=rc)
                return x, stats
        if method == "none" or stats["ve_stopped_at"] is not None:
            continue
        if frozen is not None:
            x = combine_direct(stored, frozen)
            stats["ve_steps"] += 1
            stats["frozen_steps"] += 1
            continue
        s, gamma, info = extrapolate(stored, method)
        stats["ve_steps"] += 1
        if s is None:
            stats["ve_breakdowns"] += 1
            x = stored[-1]
        else:
            stats["gammas"].append(gamma)
            stats["sum_abs_gamma"].append(info["sum_abs_gamma"])
            x = s
            if freeze_after is not None and len(stats["gammas"]) >= freeze_after:
                frozen = gamma
