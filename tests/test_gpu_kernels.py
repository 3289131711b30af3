"""Per-kernel parity of the CUDA path against the FP64 oracle, through the C-ABI, from
identical float32 inputs: the denoiser f (NLM), one FP step (Eq. (7)) for deblurring
and super-resolution, and one extrapolation (Algorithm 1 / RRE).

Tolerances (FP32 arithmetic on [0, 255] images), each an element-wise bar beside a norm
bar, so a localised error (a wrong boundary row, a wrong halo) cannot hide in the norm:
  * NLM: max |f_gpu - f_oracle| <= 2e-3 (weights come from ex2.approx, rel. error ~2^-22,
    and patch distances summed in FP32; ~1e-5 of the value range) and rel. L2 <= 1e-5;
  * one FP step (deblurring or SR): rel. L2 <= 1e-5 and max abs <= 2e-3;
  * extrapolation on the same vectors: gamma to 1e-6 relative when U is well
    conditioned; output rel. L2 <= 1e-6 and max abs <= 1e-3.
"""
import numpy as np
import pytest

from helpers import assert_step_close, f32, rel_l2, to_dev, to_host
from oracle import fp as ofp
from oracle import nlm as onlm
from oracle import operators as oops
from oracle import ve as ove
from paper_1805_02158_gb300 import red, synth

pytestmark = pytest.mark.gpu


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def deblur_problem(side_h, side_w, seed=0, psf=None):
    psf = synth.uniform_psf(9) if psf is None else psf
    return synth.make_deblur(seed, side_h, side_w, psf, 2 ** 0.5)


NLM_SIZES = [(8, 8), (48, 72), (64, 64), (96, 128), (144, 192)]
NLM_PSF = {(8, 8): synth.uniform_psf(3)}


@pytest.mark.parametrize("shape", NLM_SIZES)
def test_nlm_matches_oracle(shape):
    torch = torch_cuda()
    p = deblur_problem(*shape, psf=NLM_PSF.get(shape))
    P = red.Problem(red.config_for(p), to_dev(p.y))
    x = f32(p.y)
    f = torch.empty(shape, device="cuda")
    P.denoise(to_dev(x), f)
    torch.cuda.synchronize()
    ref = onlm.nlm(x)
    got = to_host(f)
    assert np.abs(got - ref).max() <= 2e-3
    assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("shape", [(256, 256), (1024, 1024), (192, 384)])
def test_nlm_sampled_at_full_size(shape):
    torch = torch_cuda()
    p = deblur_problem(*shape, seed=3)
    P = red.Problem(red.config_for(p), to_dev(p.y))
    x = f32(p.y)
    f = torch.empty(shape, device="cuda")
    P.denoise(to_dev(x), f)
    got = to_host(f)
    rng = np.random.default_rng(0)
    H, W = shape
    pts = [(0, 0), (H - 1, W - 1), (0, W - 1), (H - 1, 0), (H // 2, W // 2)]
    pts += [(int(rng.integers(H)), int(rng.integers(W))) for _ in range(20)]
    for (i, j) in pts:
        assert abs(got[i, j] - onlm.nlm_pixel(x, i, j)) <= 2e-3, (i, j)


def test_nlm_constant_and_shift_properties():
    torch = torch_cuda()
    p = deblur_problem(64, 64)
    P = red.Problem(red.config_for(p), to_dev(p.y))
    c = torch.full((64, 64), 93.5, device="cuda")
    f = torch.empty_like(c)
    P.denoise(c, f)
    assert float((f - 93.5).abs().max()) <= 1e-4
    x = to_dev(f32(p.y))
    f1 = torch.empty_like(x)
    f2 = torch.empty_like(x)
    P.denoise(x, f1)
    P.denoise(x + 16.0, f2)
    assert float((f2 - f1 - 16.0).abs().max()) <= 2e-3


def test_nlm_result_does_not_depend_on_the_launch_shape(monkeypatch):
    """Every NLM launch shape the autotuner chooses between (1, 2 or 4 warp tiles per CTA,
    register budget for 3 or 4 CTAs per SM; forced with RED_NLM_SHAPE) gives the same
    denoiser output and the same 12-step RRE solves bit for bit, for a single problem and
    for a batch of two sizes: the pixel-to-lane grid is fixed in image coordinates."""
    torch = torch_cuda()
    probs = [deblur_problem(64, 64, 3), deblur_problem(72, 96, 5, synth.gaussian_psf(7, 1.4))]
    ref = None
    for wy in (1, 2, 4):
        for occ in (3, 4):
            monkeypatch.setenv("RED_NLM_SHAPE", f"{wy},{occ}")
            Ps = [red.Problem(red.config_for(q, ve="rre", ve_k=5), to_dev(q.y)) for q in probs]
            x0s = [to_dev(f32(q.x0)) for q in probs]
            f = torch.empty_like(x0s[1])
            Ps[1].denoise(x0s[1], f)
            single = torch.empty_like(x0s[0])
            Ps[0].solve(x0s[0], single, 12)
            B = red.Batch(Ps)
            outs = [torch.empty_like(x) for x in x0s]
            B.solve(x0s, outs, 12, 0.0)
            shape = B.describe()
            assert (shape["nlm_warps_per_cta"], shape["nlm_ctas_per_sm"]) == (wy, occ)
            got = [to_host(f), to_host(single)] + [to_host(o) for o in outs]
            if ref is None:
                ref = got
            else:
                for a, b in zip(got, ref):
                    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("shape,psf", [((64, 64), synth.uniform_psf(9)),
                                       ((48, 72), synth.gaussian_psf(7, 1.6)),
                                       ((96, 128), synth.gaussian_psf(25, 1.6)),
                                       ((256, 256), synth.gaussian_psf(25, 1.6)),
                                       ((144, 192), synth.uniform_psf(9)),
                                       ((384, 128), synth.gaussian_psf(9, 1.2))])
def test_deblur_fp_step_matches_oracle(shape, psf):
    torch = torch_cuda()
    p = deblur_problem(*shape, psf=psf, seed=1)
    P = red.Problem(red.config_for(p), to_dev(p.y))
    x = f32(p.y)
    out = torch.empty(shape, device="cuda")
    P.fp_step(to_dev(x), out)
    ref = ofp.deblur_fp_step(x, f32(p.y), oops.psf_otf(p.psf, shape), p.sigma, p.alpha)
    assert_step_close(to_host(out), ref, f"deblur FP step {shape}")


@pytest.mark.parametrize("path", ["0", "4", "16"])
def test_deblur_fp_step_both_fourier_paths(path, monkeypatch):
    """The three-pass Fourier solve (RED_FFT_CLUSTER=0) and the cluster solve with 4 or 16
    CTAs give the oracle's FP step; includes a ragged band split (H = 72 over 16 CTAs)."""
    torch = torch_cuda()
    monkeypatch.setenv("RED_FFT_CLUSTER", path)
    for shape, psf in [((72, 96), synth.gaussian_psf(9, 1.6)), ((128, 128), synth.uniform_psf(9))]:
        p = deblur_problem(*shape, psf=psf, seed=11)
        P = red.Problem(red.config_for(p), to_dev(p.y))
        x = f32(p.y)
        out = torch.empty(shape, device="cuda")
        P.fp_step(to_dev(x), out)
        ref = ofp.deblur_fp_step(x, f32(p.y), oops.psf_otf(p.psf, shape), p.sigma, p.alpha)
        assert_step_close(to_host(out), ref, f"deblur FP step {shape}, cluster {path}")


def test_fourier_paths_agree(monkeypatch):
    """The cluster solve (16 and 4 CTAs) and the three-pass solve agree to FP32 rounding on
    the same input (same transforms, different partitions of the work)."""
    torch = torch_cuda()
    p = deblur_problem(96, 128, psf=synth.gaussian_psf(9, 1.6), seed=12)
    outs = {}
    for path in ("0", "4", "16"):
        monkeypatch.setenv("RED_FFT_CLUSTER", path)
        P = red.Problem(red.config_for(p), to_dev(p.y))
        out = torch.empty((96, 128), device="cuda")
        P.fp_step(to_dev(f32(p.y)), out)
        outs[path] = to_host(out)
    assert_step_close(outs["4"], outs["16"], "cluster 4 vs 16", rel=1e-6, max_abs=1e-3)
    assert_step_close(outs["0"], outs["16"], "three passes vs cluster 16", rel=1e-6, max_abs=1e-3)


def test_deblur_fp_step_large_uses_three_passes():
    """1024 x 1024 does not fit the cluster's shared memory: the three-pass path runs.
    Checked against the oracle's closed-form solve with f taken from the GPU denoiser
    (the oracle's own NLM is checked separately at this size by sampling)."""
    torch = torch_cuda()
    shape = (1024, 1024)
    p = deblur_problem(*shape, psf=synth.gaussian_psf(25, 1.6), seed=12)
    P = red.Problem(red.config_for(p), to_dev(p.y))
    x = to_dev(f32(p.y))
    f = torch.empty(shape, device="cuda")
    P.denoise(x, f)
    out = torch.empty(shape, device="cuda")
    P.fp_step(x, out)
    ref = ofp.deblur_solve(to_host(f), f32(p.y), oops.psf_otf(p.psf, shape), p.sigma, p.alpha)
    assert_step_close(to_host(out), ref, "1024^2 three-pass solve")


def test_deblur_linear_solve_alone_matches_closed_form():
    """x = [H^T H/s^2 + a I]^{-1}(H^T y/s^2 + a f) with f the oracle's own f(x): isolates the
    FFT solve from the denoiser."""
    torch = torch_cuda()
    p = deblur_problem(96, 128, psf=synth.gaussian_psf(25, 1.6), seed=2)
    P = red.Problem(red.config_for(p), to_dev(p.y))
    # a denoiser-free check: f(x) = x for a constant image, so the step solves with f = c
    c = np.full((96, 128), 40.0)
    out = torch.empty((96, 128), device="cuda")
    P.fp_step(to_dev(c), out)
    ref = ofp.deblur_solve(c, f32(p.y), oops.psf_otf(p.psf, (96, 128)), p.sigma, p.alpha)
    assert_step_close(to_host(out), ref, "linear solve alone")


@pytest.mark.parametrize("cluster", ["8", "10", "12", "16"])
@pytest.mark.parametrize("shape", [(48, 48), (96, 96), (54, 72)])
def test_sr_fp_step_matches_oracle(shape, cluster, monkeypatch):
    """One x3 SR FP step (NLM + 20 CG iterations), bands of 8, 10, 12 or 16 CTAs."""
    torch = torch_cuda()
    monkeypatch.setenv("RED_SR_CLUSTER", cluster)
    h, w = shape
    p = synth.make_sr(4, h, w, synth.gaussian_psf(7, 1.6), 3, 5.0)
    P = red.Problem(red.config_for(p, cg_iters=20), to_dev(p.y))
    x = f32(p.x0)
    out = torch.empty((h, w), device="cuda")
    P.fp_step(to_dev(x), out)
    ref = ofp.sr_fp_step(x, f32(p.y), oops.psf_otf(p.psf, (h, w)), 3, p.sigma, p.alpha, 20)
    assert_step_close(to_host(out), ref, f"SR FP step {shape}, cluster {cluster}")


@pytest.mark.parametrize("side,cluster", [(256, "8"), (256, "10"), (256, "12"), (256, "16"), (1024, "16"),
                                          (384, "8")])
def test_sr_linear_solve_alone_at_full_size(side, cluster, monkeypatch):
    """The CG solve alone at the workload sizes: a constant image is a fixed point of the
    denoiser (f(x) = x), so one FP step from x = c is 20 CG iterations on
    (B^T S^T S B / s^2 + a I) x = B^T S^T y / s^2 + a c, warm-started at c."""
    torch = torch_cuda()
    monkeypatch.setenv("RED_SR_CLUSTER", cluster)
    p = synth.make_sr(6, side, side, synth.gaussian_psf(7, 1.6), 3, 5.0,
                      blur=lambda x: synth.circular_blur_separable(
                          x, synth.gaussian_taps(7, 1.6), synth.gaussian_taps(7, 1.6)))
    P = red.Problem(red.config_for(p, cg_iters=20), to_dev(p.y))
    c = np.full((side, side), 80.0)
    out = torch.empty((side, side), device="cuda")
    P.fp_step(to_dev(c), out)
    ref = ofp.sr_fp_step(c, f32(p.y), oops.psf_otf(p.psf, (side, side)), 3, p.sigma, p.alpha, 20,
                         denoise=lambda v: v)
    assert_step_close(to_host(out), ref, f"SR CG alone {side}^2, cluster {cluster}")


def fp_history(p, n, kappa_plus_2):
    F = ofp.FPOperator(f32(p.y), p.psf, (p.height, p.width), p.scale, p.sigma, p.alpha)
    xs = [f32(p.x0)]
    for _ in range(n + kappa_plus_2 - 1):
        xs.append(f32(F(xs[-1])))
    return xs[n:]


@pytest.mark.parametrize("method", ["mpe", "rre", "svdmpe"])
def test_extrapolation_on_fp_history(method):
    torch = torch_cuda()
    p = deblur_problem(64, 64, seed=5)
    xs = fp_history(p, 3, 6)                 # x_3 .. x_8: kappa = 4 (ve_k = 5)
    P = red.Problem(red.config_for(p, ve=method, ve_k=5), to_dev(p.y))
    out = torch.empty((64, 64), device="cuda")
    st, gamma = P.ve_extrapolate([to_dev(x) for x in xs], out)
    x_ref, g_ref, info = ove.extrapolate(xs, method)
    assert st == red.RED_OK and not info["breakdown"]
    np.testing.assert_allclose(gamma, g_ref, rtol=1e-6, atol=1e-9)
    assert_step_close(to_host(out), x_ref, f"{method} on FP history", rel=1e-6, max_abs=1e-3)


@pytest.mark.parametrize("method", ["mpe", "rre", "svdmpe"])
def test_extrapolation_exact_on_linear_map(method):
    """A linear FP map in R^N (N = 64 x 64) with 4 distinct eigenvalues: kappa = 4 reaches
    the fixed point (Eqs. (13)-(16))."""
    torch = torch_cuda()
    rng = np.random.default_rng(1)
    n = 64 * 64
    lam = np.repeat([0.9, -0.5, 0.3, 0.7], n // 4)
    b = rng.uniform(-5, 5, n)
    x0 = rng.uniform(0, 100, n)
    xs = [x0]
    for _ in range(5):
        xs.append(lam * xs[-1] + b)
    xs32 = [f32(x).reshape(64, 64) for x in xs]
    p = deblur_problem(64, 64)
    P = red.Problem(red.config_for(p, ve=method, ve_k=5), to_dev(p.y))
    out = torch.empty((64, 64), device="cuda")
    st, gamma = P.ve_extrapolate([to_dev(x) for x in xs32], out)
    x_ref, g_ref, _ = ove.extrapolate(xs32, method)
    assert st == red.RED_OK
    np.testing.assert_allclose(gamma, g_ref, rtol=1e-5, atol=1e-8)
    assert_step_close(to_host(out), x_ref, f"{method} on a linear map", rel=1e-6, max_abs=1e-3)


def test_extrapolation_breakdown_reported():
    torch = torch_cuda()
    p = deblur_problem(64, 64)
    P = red.Problem(red.config_for(p, ve="mpe", ve_k=2), to_dev(p.y))
    v = torch.arange(64 * 64, dtype=torch.float32, device="cuda").reshape(64, 64) / 100
    xs = [v * 0, v * 1, v * 2]                # pure drift: sum c = 0
    out = torch.empty_like(v)
    st, gamma = P.ve_extrapolate(xs, out)
    assert st == red.RED_EVE_BREAKDOWN and gamma is None
    assert float((out - xs[-1]).abs().max()) == 0.0



def _integer_history(dep):
    """Five iterates x_0 .. x_4 on an integer grid (exact in float32, and so their
    differences and the Gram entries), whose differences u_0 .. u_3 carry one exact linear
    dependency: "early" u_1 = u_0 (rank loss in the first kappa columns), "last"
    u_3 = u_0 - u_1 (rank loss in the last column only)."""
    rng = np.random.default_rng(7)
    n = 64 * 64
    u = [rng.integers(-8, 9, n).astype(np.float64) for _ in range(3)]
    if dep == "early":
        u = [u[0], u[0].copy(), u[1], u[2]]
    else:
        u = [u[0], u[1], u[2], u[0] - u[1]]
    xs = [rng.integers(50, 150, n).astype(np.float64)]
    for d in u:
        xs.append(xs[-1] + d)
    return [x.astype(np.float32).reshape(64, 64) for x in xs]


@pytest.mark.parametrize("method", ["mpe", "rre", "svdmpe"])
def test_extrapolation_rank_loss_in_an_early_column_is_a_breakdown(method):
    """A dependent column among the first kappa (Algorithm 2's r_jj = 0) leaves gamma
    undefined for every method: breakdown, the last iterate returned, as the oracle."""
    torch = torch_cuda()
    xs = _integer_history("early")
    _, g_ref, info = ove.extrapolate([f32(x) for x in xs], method)
    assert info["breakdown"] and g_ref is None
    p = deblur_problem(64, 64)
    P = red.Problem(red.config_for(p, ve=method, ve_k=4), to_dev(p.y))
    out = torch.empty((64, 64), device="cuda")
    st, gamma = P.ve_extrapolate([to_dev(x) for x in xs], out)
    assert st == red.RED_EVE_BREAKDOWN and gamma is None
    np.testing.assert_array_equal(to_host(out), xs[-1])


@pytest.mark.parametrize("method", ["mpe", "rre", "svdmpe"])
def test_extrapolation_rank_loss_in_the_last_column(method):
    """u_3 = u_0 - u_1 exactly: MPE (Algorithm 1 uses only R's leading kappa columns and
    its last column) gives c = (-1, 1, 0, 1), RRE falls back to MPE (Eq. (19) needs all of
    R), and SVD-MPE takes the null vector of R; all three as the oracle, and the combination
    sum gamma_i x_i is the exact fixed point of the dependency."""
    torch = torch_cuda()
    xs = _integer_history("last")
    x_ref, g_ref, info = ove.extrapolate([f32(x) for x in xs], method)
    assert not info["breakdown"] and info["rank_deficient"] == [3]
    np.testing.assert_allclose(g_ref, [-1.0, 1.0, 0.0, 1.0], atol=1e-9)
    p = deblur_problem(64, 64)
    P = red.Problem(red.config_for(p, ve=method, ve_k=4), to_dev(p.y))
    out = torch.empty((64, 64), device="cuda")
    st, gamma = P.ve_extrapolate([to_dev(x) for x in xs], out)
    assert st == red.RED_OK
    np.testing.assert_allclose(gamma, g_ref, rtol=1e-6, atol=1e-9)
    assert_step_close(to_host(out), x_ref, f"{method}, rank loss in the last column", rel=1e-6,
                      max_abs=1e-3)

def test_measured_unit_peaks_are_plausible():
    """The arithmetic-unit microbenchmarks: FP32 FMA near 152 SMs x 128 lanes x clock, the
    special-function unit a fraction of it, FP64 far below FP32 on this part."""
    torch_cuda()
    m = red.measure_peaks()
    assert 5e12 < m["fp32_fma"] < 60e12
    assert 0 < m["ex2"] < m["fp32_fma"]
    assert 0 < m["fp64_fma"] < m["fp32_fma"]
