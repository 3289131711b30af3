"""GPU parity cases outside the paper's settings: PSFs that are not symmetric (the paper's
are), where the conjugate of the PSF spectrum in H^T (Eq. (7)) and the orientation of the
taps in the SR passes matter, and the largest accepted image side (2048).

Bars as in test_gpu_kernels.py: one FP step (deblurring, or SR with 20 CG iterations)
within 1e-5 relative L2 and 2e-3 max abs of the oracle, NLM samples within 2e-3 on
[0, 255]."""
import numpy as np
import pytest

from helpers import assert_step_close, f32, to_dev, to_host
from oracle import fp as ofp
from oracle import nlm as onlm
from oracle import operators as oops
from paper_1805_02158_gb300 import red, synth

pytestmark = pytest.mark.gpu


def asymmetric_psf(kh, kw, seed):
    """Random non-negative taps summing to 1, no symmetry (a complex PSF spectrum)."""
    a = np.random.default_rng(seed).uniform(0.0, 1.0, (kh, kw))
    a[0, kw - 1] += 2.0          # a strong off-centre tap: orientation errors are large
    return a / a.sum()


@pytest.mark.parametrize("path", ["0", "16"])
def test_asymmetric_psf_deblur_fp_step(path, monkeypatch):
    import torch
    monkeypatch.setenv("RED_FFT_CLUSTER", path)
    psf = asymmetric_psf(5, 7, 1)
    p = synth.make_deblur(21, 72, 96, psf, 2 ** 0.5)
    P = red.Problem(red.config_for(p), to_dev(p.y))
    x = f32(p.y)
    out = torch.empty((72, 96), device="cuda")
    P.fp_step(to_dev(x), out)
    ref = ofp.deblur_fp_step(x, f32(p.y), oops.psf_otf(f32(psf), (72, 96)), p.sigma, p.alpha)
    assert_step_close(to_host(out), ref, f"asymmetric PSF deblur, cluster {path}")


@pytest.mark.parametrize("kh,kw", [(7, 7), (5, 9)])
def test_asymmetric_psf_sr_fp_step(kh, kw):
    """7x7 takes the compile-time x3 / 7x7 kernel, 5x9 the generic one."""
    import torch
    psf = asymmetric_psf(kh, kw, 2)
    p = synth.make_sr(22, 48, 48, psf, 3, 5.0)
    P = red.Problem(red.config_for(p, cg_iters=20), to_dev(p.y))
    x = f32(p.x0)
    out = torch.empty((48, 48), device="cuda")
    P.fp_step(to_dev(x), out)
    ref = ofp.sr_fp_step(x, f32(p.y), oops.psf_otf(f32(psf), (48, 48)), 3, p.sigma, p.alpha, 20)
    assert_step_close(to_host(out), ref, f"asymmetric PSF SR {kh}x{kw}")


def test_largest_side_deblur():
    """2048 x 2048: NLM sampled against the per-pixel definition, and the Fourier solve
    alone (a constant image is a fixed point of the denoiser) against the oracle."""
    import torch
    side = 2048
    p = synth.make_deblur(23, side, side, synth.uniform_psf(9), 2 ** 0.5)
    P = red.Problem(red.config_for(p), to_dev(p.y))
    x = f32(p.y)
    f = torch.empty((side, side), device="cuda")
    P.denoise(to_dev(x), f)
    fh = to_host(f)
    for i, j in [(0, 0), (0, side - 1), (side - 1, 0), (side - 1, side - 1), (1023, 1500), (7, 2041)]:
        assert abs(fh[i, j] - onlm.nlm_pixel(x, i, j)) <= 2e-3
    c = np.full((side, side), 60.0)
    out = torch.empty((side, side), device="cuda")
    P.fp_step(to_dev(c), out)
    ref = ofp.deblur_solve(c, f32(p.y), oops.psf_otf(p.psf, (side, side)), p.sigma, p.alpha)
    assert_step_close(to_host(out), ref, "2048^2 deblur solve")


def test_largest_side_sr():
    """2048 x 2048 x3 SR: the CG solve alone from a constant image (bands stream from L2)."""
    import torch
    side = 2048
    taps = synth.gaussian_taps(7, 1.6)
    p = synth.make_sr(24, side, side, synth.gaussian_psf(7, 1.6), 3, 5.0,
                      blur=lambda v: synth.circular_blur_separable(v, taps, taps))
    P = red.Problem(red.config_for(p, cg_iters=20), to_dev(p.y))
    c = np.full((side, side), 80.0)
    out = torch.empty((side, side), device="cuda")
    P.fp_step(to_dev(c), out)
    ref = ofp.sr_fp_step(c, f32(p.y), oops.psf_otf(p.psf, (side, side)), 3, p.sigma, p.alpha, 20,
                         denoise=lambda v: v)
    assert_step_close(to_host(out), ref, "2048^2 SR CG alone")
