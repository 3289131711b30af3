"""Writes tests/golden/full_size_oracle.json and tests/golden/full_size_oracle.npz: FP64
oracle solves of the full-size workloads at the paper's budget of 200 FP steps (denoiser
calls; Tables I and II compare the methods after 200 FP iterations, Sec. IV-A/B), from
oracle/ and the input generators only. Nothing here comes from the CUDA path.

Cases:
  * deblurring, 256x256, 25x25 Gaussian PSF (std 1.6), noise sqrt 2 (Sec. IV-A;
    synth.deblur_gauss256): RRE with ve_k = 5 (kappa = 4) on seeds 0-9 (the ten images of
    the benchmark batch); MPE k = 5, RRE k = 10, MPE k = 10, SVD-MPE k = 5 and plain FP on
    seeds 0 and 7;
  * x3 super-resolution, 256x256 HR, 7x7 Gaussian (std 1.6), noise 5, CG 20 (Sec. IV-B;
    synth.sr_x3): RRE k = 5 on seeds 0-2; MPE k = 5 and plain FP on seed 0.

Per case: the iterates after 20 and after 200 calls (float32 in the .npz, keys
"<case>@20" and "<case>"), the final PSNR against the ground truth, the objective E(x) of
Eq. (4), the solve's counters and, for the traced cases (seed 0 of plain FP, RRE k = 5 and
MPE k = 5 of both tasks), for every FP step the fixed-point residual ||F(x) - x|| / ||x||
at the point it starts from, whether that point was an extrapolated vector, and E(x) at
that point (from the step's own f(x)); and the objective of the FP iterate after every 5
calls (Table I's criterion).

Sensitivity of the method itself: every case is solved again with each FP step's output
rounded to 20 significant bits (relative rounding 2^-21, rms about 2.8e-7: the relative L2
size of the per-step error the FP32 GPU path makes, measured 2.2e-7 - 3.3e-7 per FP step
against this oracle) and to 19 bits (2^-20: the size of its largest per-pixel errors,
2-3e-4 on values near 100), and the distance of each such solve from the FP64 one
(relative L2, |PSNR difference|, max abs) is stored at 20 and 200 calls under
"sensitivity" -> "<bits>".
Extrapolation combines the iterates with weights whose absolute sum sum |gamma_i|
(Eq. (21)) bounds how much a perturbation of them is magnified; near convergence the
columns of U are nearly dependent, sum |gamma| reaches 10^2 - 10^6, and over 40 cycles the
magnification compounds, so this distance is what any implementation with per-step
errors of that size must be expected to show.

Usage: python tests/golden/make_full_size_oracle.py [--workers N]   (about 45 minutes on
8 cores); --add-sensitivity BITS recomputes only the BITS-bit realization of the stored
cases (about 15 minutes).
"""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")   # one thread per worker process

import argparse  # noqa: E402
import json  # noqa: E402
import multiprocessing as mp  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CALLS = 200
EARLY = 20          # the early budget also stored (4 cycles of k = 5, 2 of k = 10)
SENS_BITS = (20, 19)   # significant bits of the perturbed solves' iterates
JSON_PATH = os.path.join(HERE, "full_size_oracle.json")
NPZ_PATH = os.path.join(HERE, "full_size_oracle.npz")

TRACED = {"deblur256_none_k5_s0", "deblur256_rre_k5_s0", "deblur256_mpe_k5_s0",
          "sr256_none_k5_s0", "sr256_rre_k5_s0", "sr256_mpe_k5_s0"}


def case_list():
    """(name, task, seed, method, ve_k)."""
    out = [(f"deblur256_rre_k5_s{s}", "deblur", s, "rre", 5) for s in range(10)]
    for s in (0, 7):
        for method, k in (("mpe", 5), ("rre", 10), ("mpe", 10), ("svdmpe", 5), ("none", 5)):
            out.append((f"deblur256_{method}_k{k}_s{s}", "deblur", s, method, k))
    out += [(f"sr256_rre_k5_s{s}", "sr", s, "rre", 5) for s in range(3)]
    out += [("sr256_mpe_k5_s0", "sr", 0, "mpe", 5), ("sr256_none_k5_s0", "sr", 0, "none", 5)]
    return out


def problem(task, seed):
    from paper_1805_02158_gb300 import synth
    return synth.deblur_gauss256(seed) if task == "deblur" else synth.sr_x3(seed)


class Traced:
    """The FP map with a record of every evaluation: residual and objective at its input."""

    def __init__(self, F):
        self.F = F
        self.residual, self.objective, self.inputs = [], [], []

    def __call__(self, x):
        from oracle import red
        xn, f = self.F.step_with_f(x)
        self.residual.append(float(np.linalg.norm(xn - x) / np.linalg.norm(x)))
        self.objective.append(red.objective(x, f, self.F.y, self.F.otf, self.F.scale,
                                            self.F.sigma, self.F.alpha))
        self.inputs.append(x)
        return xn


def round_bits(x, bits):
    """x rounded to `bits` significant bits (round half to even), elementwise."""
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 2.0 ** bits) / 2.0 ** bits, e)


class Rounded:
    """The FP map with its output rounded to `bits` significant bits."""

    def __init__(self, F, bits):
        self.F, self.bits = F, bits

    def __call__(self, x):
        return round_bits(self.F(x), self.bits)


def distance(x, ref, x_true):
    from oracle import red
    return {"rel_l2": float(np.linalg.norm(x - ref) / np.linalg.norm(ref)),
            "psnr_db": float(abs(red.psnr(x, x_true) - red.psnr(ref, x_true))),
            "max_abs": float(np.abs(x - ref).max())}


def perturbed(case, bits, x_ref, x_ref_early):
    """Distance from the FP64 solve of the solve whose FP outputs are rounded to `bits`
    significant bits, at EARLY and CALLS calls."""
    from oracle import fp, red
    name, task, seed, method, k = case
    p = problem(task, seed)
    y = np.asarray(p.y, np.float32).astype(np.float64)
    x0 = np.asarray(p.x0, np.float32).astype(np.float64)
    F = fp.FPOperator(y, p.psf, (p.height, p.width), p.scale, p.sigma, p.alpha)
    early = {}

    def cb(calls, xp):
        if calls == EARLY:
            early["x"] = xp.copy()

    xp, _ = red.solve(Rounded(F, bits), x0, method, m=0, kappa=k - 1, max_calls=CALLS,
                      callback=cb)
    return {"at_200": distance(xp, x_ref, p.x_true),
            "at_20": distance(early["x"], x_ref_early, p.x_true)}


def add_sensitivity(task_args):
    """(case, bits) -> (name, bits, distances) for a stored case."""
    case, bits = task_args
    with np.load(NPZ_PATH) as z:
        x_ref = z[case[0]].astype(np.float64)
        x_early = z[f"{case[0]}@{EARLY}"].astype(np.float64)
    return case[0], bits, perturbed(case, bits, x_ref, x_early)


def run_case(case):
    from oracle import fp, red
    name, task, seed, method, k = case
    t0 = time.time()
    p = problem(task, seed)
    y = np.asarray(p.y, np.float32).astype(np.float64)
    x0 = np.asarray(p.x0, np.float32).astype(np.float64)
    F = fp.FPOperator(y, p.psf, (p.height, p.width), p.scale, p.sigma, p.alpha)
    traced = name in TRACED
    G = Traced(F) if traced else F
    every5 = []
    outputs = []
    early = {}

    def cb(calls, x):
        if calls == EARLY:
            early["x"] = x.copy()
        if traced:
            outputs.append(x)
        if traced and calls % 5 == 0:
            every5.append(red.objective(x, F.denoise(x), F.y, F.otf, F.scale, F.sigma, F.alpha))

    x, st = red.solve(G, x0, method, m=0, kappa=k - 1, max_calls=CALLS, callback=cb)
    sens = {str(b): perturbed(case, b, x, early["x"]) for b in SENS_BITS}
    e = red.objective(x, F.denoise(x), F.y, F.otf, F.scale, F.sigma, F.alpha)
    rec = {"task": task, "seed": seed, "method": method, "ve_k": k, "kappa": k - 1, "m": 0,
           "calls": CALLS, "fp_calls": st["fp_calls"], "ve_steps": st["ve_steps"],
           "ve_breakdowns": st["ve_breakdowns"],
           "sum_abs_gamma_max": max(st["sum_abs_gamma"]) if st["sum_abs_gamma"] else None,
           "psnr": red.psnr(x, p.x_true), "objective": e,
           "sensitivity": sens}
    if traced:
        # a call's input is an extrapolated vector when it is not the previous call's output
        extrap = [False] + [not np.array_equal(G.inputs[i], outputs[i - 1])
                            for i in range(1, len(G.inputs))]
        rec["trace"] = {"residual_at_input": G.residual, "objective_at_input": G.objective,
                        "input_is_extrapolated": extrap, "objective_every5": every5}
    rec["seconds"] = time.time() - t0
    return name, rec, x.astype(np.float32), early["x"].astype(np.float32)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--add-sensitivity", type=int, default=0)
    args = ap.parse_args()
    cases = case_list()
    if args.add_sensitivity:
        # the stored iterates are float32 roundings of the FP64 solves: the distances of a
        # perturbed solve from them differ from those to the FP64 solve by < 1e-7 relative
        cases.sort(key=lambda c: c[1] != "sr")
        with mp.get_context("spawn").Pool(args.workers) as pool:
            res = pool.map(add_sensitivity, [(c, args.add_sensitivity) for c in cases], chunksize=1)
        out = json.load(open(JSON_PATH))
        for name, bits, d in res:
            out["cases"][name]["sensitivity"][str(bits)] = d
        with open(JSON_PATH, "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        print(f"added the {args.add_sensitivity}-bit realization to {len(res)} cases")
        return
    # longest first: the traced and super-resolution cases
    cases.sort(key=lambda c: (c[0] not in TRACED, c[1] != "sr"))
    with mp.get_context("spawn").Pool(args.workers) as pool:
        results = pool.map(run_case, cases, chunksize=1)
    out = {"_source": "written by tests/golden/make_full_size_oracle.py from oracle/ only",
           "_budget": "200 FP steps per solve (Sec. IV-A/B, Tables I and II)",
           "cases": {}}
    arrays = {}
    for name, rec, x, x20 in sorted(results, key=lambda r: r[0]):
        out["cases"][name] = rec
        arrays[name] = x
        arrays[f"{name}@{EARLY}"] = x20
    with open(JSON_PATH, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    np.savez_compressed(NPZ_PATH, **arrays)
    print(f"wrote {len(results)} cases")


if __name__ == "__main__":
    main()
