"""The experimental settings the paper prints (Sec. IV-A, IV-B, IV-C; Tables I and II),
stored with their citations in tests/golden/paper_settings.json, against the synthetic
problem generators and the benchmark's configuration."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1805_02158_gb300 import synth  # noqa: E402

GOLDEN = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_settings.json")))


def second_moment(psf):
    """Variance of the PSF along its first axis about the centre (psf sums to 1)."""
    k = psf.shape[0]
    a = np.arange(k) - (k - 1) / 2
    return float((psf.sum(axis=1) * a ** 2).sum())


def test_deblurring_problems_use_the_paper_physics():
    g = GOLDEN["deblur"]
    p = synth.deblur_small(0)
    k = g["uniform_psf_size"]
    assert p.psf.shape == (k, k) and np.allclose(p.psf, 1.0 / (k * k))
    assert p.sigma == pytest.approx(g["noise_sigma"], rel=1e-15) and p.scale == 1
    q = synth.deblur_gauss256(0, 64)
    assert q.sigma == pytest.approx(g["noise_sigma"], rel=1e-15)
    # 25x25 support: truncation at +-7.5 std leaves the variance at std^2
    assert abs(q.psf.sum() - 1.0) < 1e-12 and np.allclose(q.psf, q.psf.T)
    assert second_moment(q.psf) == pytest.approx(g["gaussian_psf_std"] ** 2, rel=1e-9)


def test_super_resolution_problems_use_the_paper_physics():
    g = GOLDEN["super_resolution"]
    p = synth.sr_x3(0, 48)
    assert p.scale == g["scale"] and p.sigma == g["noise_sigma"]
    assert p.psf.shape == (g["gaussian_psf_size"],) * 2
    assert np.allclose(p.psf, synth.gaussian_psf(g["gaussian_psf_size"], g["gaussian_psf_std"]))
    # on 7 taps the Gaussian is cut at +-3 (1.9 std): the variance is below std^2, and
    # equals the truncated sum computed here from the taps' definition
    a = np.arange(7) - 3.0
    w = np.exp(-a ** 2 / (2 * g["gaussian_psf_std"] ** 2))
    assert second_moment(p.psf) == pytest.approx(float((w * a ** 2).sum() / w.sum()), rel=1e-12)
    assert p.y.shape == (48 // 3, 48 // 3)


def test_benchmark_budgets_and_robustness_grid_follow_the_paper():
    import bench
    assert bench.CALLS == GOLDEN["table_1_deblur_calls"]["fp"] == GOLDEN["table_2_sr_calls"]["fp"]
    grid = GOLDEN["robustness_grid"]
    assert list(bench.SWEEP_M) == grid["m"] and list(bench.SWEEP_KAPPA) == grid["kappa"]
    lo, hi = grid["search_range"]
    assert all(lo <= v <= hi for v in bench.SWEEP_M + bench.SWEEP_KAPPA)
    assert min(bench.SWEEP_KAPPA) >= grid["kappa_min"]


def test_table_counts_support_five_fp_steps_per_cycle():
    """Every FP-MPE count of Tables I and II is a multiple of 5, the paper's printed kappa
    for FP-MPE: read as 5 FP steps (denoiser calls) per cycle, which is the benchmark's
    extrapolation setting ve_k = 5."""
    import bench
    counts = (list(GOLDEN["table_1_deblur_calls"]["uniform"].values())
              + list(GOLDEN["table_1_deblur_calls"]["gaussian"].values())
              + list(GOLDEN["table_2_sr_calls"]["counts"].values()))
    assert len(counts) == 29
    assert all(c % 5 == 0 for c in counts)
    assert GOLDEN["deblur"]["fp_mpe_kappa"] == GOLDEN["super_resolution"]["fp_mpe_kappa"] == bench.VE_K
    assert max(counts) < GOLDEN["table_1_deblur_calls"]["fp"]
