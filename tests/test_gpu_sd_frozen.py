"""GPU parity of the two variants of Algorithm 3 that the paper evaluates besides FP-MPE/RRE,
against the FP64 oracle, through the C-ABI:

  * SD-MPE (Sec. IV-A, Sec. IV-B): the baseline map is the fixed-step steepest descent
    x - mu grad E(x) on Eq. (5) (oracle/sd.py) instead of the FP step of Eq. (7); the paper
    runs MPE on it with m = 0, kappa = 8 for deblurring and m = 1, kappa = 10 for x3 SR;
  * cycling with frozen gamma (a remark of Sec. III-C): after n successful extrapolations
    later cycles run m + kappa baseline steps and combine with the last gamma
    (oracle/red.py solve(..., freeze_after=n)).

Bars: one SD step as one FP step (relative L2 <= 1e-5, max abs <= 2e-3); solves to the FP32
solve bars (relative L2 <= 1e-3, |PSNR difference| <= 0.01 dB, max abs <= 0.5), or, for
SD-MPE, whose steepest-descent iterates move along nearly one direction so that MPE's
weights reach sum |gamma| ~ 10^5 - 10^6 (Eq. (21)), within 3x the oracle's own response to
per-step perturbations of the FP32 path's size (helpers.solve_bars)."""
import numpy as np
import pytest

from helpers import (assert_solve_close, assert_step_close, f32, oracle_sensitivity, solve_bars,
                     to_dev, to_host)
from oracle import fp as ofp
from oracle import red as ored
from oracle import sd as osd
from paper_1805_02158_gb300 import red, synth

pytestmark = pytest.mark.gpu


def sd_map(p, mu=None):
    return osd.SDOperator(f32(p.y), p.psf, (p.height, p.width), p.scale, p.sigma, p.alpha, mu=mu)


def fp_map(p):
    return ofp.FPOperator(f32(p.y), p.psf, (p.height, p.width), p.scale, p.sigma, p.alpha)


def gpu_solve(p, calls, **cfg):
    import torch
    P = red.Problem(red.config_for(p, **cfg), to_dev(p.y))
    out = torch.empty((p.height, p.width), device="cuda")
    st = P.solve(to_dev(f32(p.x0)), out, calls, 0.0)
    return to_host(out), st


@pytest.mark.parametrize("path", ["0", "16"])
def test_sd_step_deblur_both_fourier_paths(path, monkeypatch):
    import torch
    monkeypatch.setenv("RED_FFT_CLUSTER", path)
    p = synth.make_deblur(31, 72, 96, synth.gaussian_psf(9, 1.6), 2 ** 0.5)
    P = red.Problem(red.config_for(p, baseline="sd"), to_dev(p.y))
    x = f32(p.y)
    out = torch.empty((72, 96), device="cuda")
    P.fp_step(to_dev(x), out)
    assert_step_close(to_host(out), sd_map(p)(x), f"SD step deblur, cluster {path}")


@pytest.mark.parametrize("kh,kw", [(7, 7), (5, 9)])
def test_sd_step_sr(kh, kw):
    """7x7 takes the compile-time x3 / 7x7 kernel, 5x9 the generic one."""
    import torch
    psf = synth.gaussian_psf(7, 1.6) if kh == 7 else np.outer(synth.gaussian_taps(5, 1.2),
                                                               synth.gaussian_taps(9, 1.8))
    p = synth.make_sr(32, 48, 48, psf / psf.sum(), 3, 5.0)
    P = red.Problem(red.config_for(p, baseline="sd"), to_dev(p.y))
    x = f32(p.x0)
    out = torch.empty((48, 48), device="cuda")
    P.fp_step(to_dev(x), out)
    assert_step_close(to_host(out), sd_map(p)(x), f"SD step SR {kh}x{kw}")


def test_sd_step_with_given_mu():
    import torch
    p = synth.deblur_small(3)
    mu = 0.5 * osd.default_step(sd_map(p).otf, p.sigma, p.alpha)
    P = red.Problem(red.config_for(p, baseline="sd", sd_mu=mu), to_dev(p.y))
    x = f32(p.y)
    out = torch.empty((64, 64), device="cuda")
    P.fp_step(to_dev(x), out)
    assert_step_close(to_host(out), sd_map(p, mu)(x), "SD step, given mu")


def _sd_mpe_case(p, m, kappa, calls, label):
    x_ref, st_ref = ored.solve(sd_map(p), f32(p.x0), "mpe", m=m, kappa=kappa, max_calls=calls)
    sens = oracle_sensitivity(lambda: sd_map(p), f32(p.x0), x_ref, p.x_true, "mpe", m, kappa,
                              calls)
    x, st = gpu_solve(p, calls, baseline="sd", ve="mpe", ve_k=kappa + 1, ve_m=m)
    assert st["fp_calls"] == calls and st["ve_steps"] == st_ref["ve_steps"]
    rel, db, ma = solve_bars(sens)
    assert_solve_close(x, x_ref, p.x_true, f"{label} (oracle sensitivity {sens})", rel=rel, db=db,
                       max_abs=ma)


def test_sd_mpe_deblur_paper_setting():
    """SD-MPE with the paper's deblurring setting (m = 0, kappa = 8: ve_k = 9): two cycles
    (18 calls) and 40 calls."""
    p = synth.deblur_small(5)
    _sd_mpe_case(p, 0, 8, 18, "SD-MPE deblur m=0 kappa=8, 18 calls")
    _sd_mpe_case(p, 0, 8, 40, "SD-MPE deblur m=0 kappa=8, 40 calls")


def test_sd_mpe_sr_paper_setting():
    """SD-MPE with the paper's x3 SR setting (m = 1, kappa = 10: ve_k = 11), 36 calls."""
    _sd_mpe_case(synth.sr_x3(3, 72), 1, 10, 36, "SD-MPE SR m=1 kappa=10")


def test_plain_sd_matches_oracle():
    p = synth.deblur_small(6)
    F = sd_map(p)
    x_ref = f32(p.x0)
    for _ in range(25):
        x_ref = F(x_ref)
    x, st = gpu_solve(p, 25, baseline="sd", ve="none")
    assert st["fp_calls"] == 25
    assert_solve_close(x, x_ref, p.x_true, "plain SD, 25 steps")


@pytest.mark.parametrize("method,k,m,freeze,calls", [("rre", 5, 0, 2, 40), ("mpe", 4, 1, 1, 31),
                                                     ("rre", 3, 0, 1, 30)])
def test_frozen_gamma_deblur_matches_oracle(method, k, m, freeze, calls):
    p = synth.deblur_small(7)
    x_ref, st_ref = ored.solve(fp_map(p), f32(p.x0), method, m=m, kappa=k - 1, max_calls=calls,
                               freeze_after=freeze)
    assert st_ref["frozen_steps"] > 0
    x, st = gpu_solve(p, calls, ve=method, ve_k=k, ve_m=m, ve_freeze=freeze)
    assert st["fp_calls"] == calls
    assert st["ve_steps"] == st_ref["ve_steps"], (st, st_ref)
    assert_solve_close(x, x_ref, p.x_true, f"frozen gamma {method} k={k} m={m} after {freeze}")


def test_frozen_gamma_sr_matches_oracle():
    p = synth.sr_x3(4, 48)
    x_ref, st_ref = ored.solve(fp_map(p), f32(p.x0), "rre", m=0, kappa=4, max_calls=27,
                               freeze_after=1)
    x, st = gpu_solve(p, 27, ve="rre", ve_k=5, ve_freeze=1)
    assert st["fp_calls"] == 27 and st["ve_steps"] == st_ref["ve_steps"]
    assert_solve_close(x, x_ref, p.x_true, "frozen gamma SR")


def test_frozen_sd_mpe_and_mixed_baselines_batch_equal_single_solves():
    """A batch mixing FP and SD problems, with frozen gamma, reproduces each problem's
    single solve bit for bit."""
    import torch
    probs = [synth.deblur_small(8), synth.make_deblur(9, 48, 72, synth.gaussian_psf(7, 1.6), 2.0),
             synth.deblur_small(10)]
    kws = [dict(baseline="sd"), dict(baseline="fp"), dict(baseline="sd")]
    common = dict(ve="mpe", ve_k=5, ve_freeze=2)
    singles = [gpu_solve(p, 33, **common, **kw)[0] for p, kw in zip(probs, kws)]
    Ps = [red.Problem(red.config_for(p, **common, **kw), to_dev(p.y)) for p, kw in zip(probs, kws)]
    B = red.Batch(Ps)
    x0s = [to_dev(f32(p.x0)) for p in probs]
    outs = [torch.empty_like(x) for x in x0s]
    stats = B.solve(x0s, outs, 33, 0.0)
    for s, o, ref in zip(stats, outs, singles):
        assert s["fp_calls"] == 33
        np.testing.assert_array_equal(to_host(o), ref)
