"""GPU solves at the paper's budget of 200 FP steps (Tables I and II, Sec. IV-A/B) against
the FP64 oracle's solves of the same problems, stored in tests/golden/full_size_oracle.*
by tests/golden/make_full_size_oracle.py (oracle/ only).

  * the benchmark batch exactly as bench.py times it: ten 256x256 deblurring problems
    (25x25 Gaussian PSF std 1.6, noise sqrt 2), RRE with ve_k = 5, one red.Batch with the
    autotuned launch shapes, x0 = y, 200 FP steps; every image to the FP32 solve bars
    (relative L2 <= 1e-3, |PSNR difference| <= 0.01 dB, every pixel within 0.5 grey
    levels) and the same extrapolation counts as the oracle;
  * MPE k = 5, RRE k = 10, MPE k = 10, SVD-MPE k = 5 and plain FP on images 0 and 7;
  * x3 super-resolution (256x256 HR, CG 20), RRE k = 5 on images 0-2 in FP32 storage to the
    same bars, and in BF16 and FP16 storage with their errors stated (PSNR, relative L2,
    max abs).
"""
import json
import os

import numpy as np
import pytest

from helpers import assert_solve_close, f32, solve_errors, to_dev, to_host
from paper_1805_02158_gb300 import red, synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CASES = json.load(open(os.path.join(GOLDEN, "full_size_oracle.json")))["cases"]
CALLS = 200


def stored(name):
    with np.load(os.path.join(GOLDEN, "full_size_oracle.npz")) as z:
        return z[name].astype(np.float64)


def batch_solve(probs, method, k, storage="f32"):
    import torch
    ys = [to_dev(p.y) for p in probs]
    Ps = [red.Problem(red.config_for(p, ve=method, ve_k=k, storage=storage), y)
          for p, y in zip(probs, ys)]
    B = red.Batch(Ps)
    x0s = [to_dev(f32(p.x0)) for p in probs]
    outs = [torch.empty_like(x) for x in x0s]
    stats = B.solve(x0s, outs, CALLS, 0.0)
    return [to_host(o) for o in outs], stats


def check_counts(st, ref):
    assert st["fp_calls"] == ref["fp_calls"] == CALLS
    assert st["ve_steps"] == ref["ve_steps"]
    assert st["ve_breakdowns"] == ref["ve_breakdowns"]


def test_benchmark_batch_at_200_calls():
    probs = [synth.deblur_gauss256(s) for s in range(10)]
    xs, stats = batch_solve(probs, "rre", 5)
    worst = {"rel_l2": 0.0, "psnr_db": 0.0, "max_abs": 0.0}
    for s, (x, st, p) in enumerate(zip(xs, stats, probs)):
        name = f"deblur256_rre_k5_s{s}"
        check_counts(st, CASES[name])
        e = assert_solve_close(x, stored(name), p.x_true, f"benchmark batch image {s}")
        worst = {k: max(worst[k], e[k]) for k in worst}
    print(f"benchmark batch, worst of 10 images: {worst}")


@pytest.mark.parametrize("method,k", [("mpe", 5), ("rre", 10), ("mpe", 10), ("svdmpe", 5),
                                      ("none", 5)])
def test_deblur_variants_at_200_calls(method, k):
    probs = [synth.deblur_gauss256(s) for s in (0, 7)]
    xs, stats = batch_solve(probs, method, k)
    for s, x, st, p in zip((0, 7), xs, stats, probs):
        name = f"deblur256_{method}_k{k}_s{s}"
        check_counts(st, CASES[name])
        assert_solve_close(x, stored(name), p.x_true,
                           f"{name} (oracle max sum|gamma| {CASES[name]['sum_abs_gamma_max']})")


def test_sr_at_200_calls_f32():
    probs = [synth.sr_x3(s) for s in range(3)]
    xs, stats = batch_solve(probs, "rre", 5)
    for s, x, st, p in zip(range(3), xs, stats, probs):
        name = f"sr256_rre_k5_s{s}"
        check_counts(st, CASES[name])
        assert_solve_close(x, stored(name), p.x_true, f"{name} f32")


# (PSNR dB, relative L2, max abs on [0, 255]) bounds of 16-bit storage over a 200-step SR
# solve: BF16 as in the 20-step full-size test, FP16 (3 more significant bits) 8x tighter
BOUNDS_16 = {"bf16": (0.25, 1e-2, 32.0), "f16": (0.03, 1.25e-3, 4.0)}


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_sr_at_200_calls_16_bit_error_stated(storage):
    """16-bit storage of the iterates (FP32 arithmetic): the errors against the FP64 oracle
    are stated per image and bounded."""
    probs = [synth.sr_x3(s) for s in range(3)]
    xs, stats = batch_solve(probs, "rre", 5, storage=storage)
    db, rel, ma = BOUNDS_16[storage]
    for s, x, st, p in zip(range(3), xs, stats, probs):
        name = f"sr256_rre_k5_s{s}"
        e = solve_errors(x, stored(name), p.x_true)
        print(f"{name} {storage} storage: PSNR error {e['psnr_db']:.4f} dB, relative L2 "
              f"{e['rel_l2']:.3e}, max abs {e['max_abs']:.3f}")
        assert e["psnr_db"] <= db and e["rel_l2"] <= rel and e["max_abs"] <= ma, e
