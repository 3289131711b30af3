"""The allocation-free extrapolation entry point (red_ve_extrapolate_static) against the
problem-based one (red_ve_extrapolate) on the same device vectors.

Both evaluate the same Gram matrix with exact products and double-float sums (reduced in
different orders: a grid-strided fixed-size scratch here, one row per chunk there), the
same double-word solve and the same combine. Their G then differ in the last double-word
bits (~2^-48 relative), which the solve maps to gamma with a factor of cond(G); the cases
below include a deliberately near-singular G (four differences of a map with three
distinct eigenvalues), so gamma is compared at rtol 1e-8 (GAMMA_RTOL), still far below the
float32 rounding of the xi that the combine consumes, and the outputs to a few float32 ulps
(max abs <= 1e-4 on [0, 255] images). This file is collected last so that the static scratch is exercised after the
other GPU tests have used the device.
"""
import ctypes

import numpy as np
import pytest

from helpers import f32, to_dev
from oracle import fp as ofp
from paper_1805_02158_gb300 import red, synth

pytestmark = pytest.mark.gpu

GAMMA_RTOL = 1e-8


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def fp_history(p, n, count):
    F = ofp.FPOperator(f32(p.y), p.psf, (p.height, p.width), p.scale, p.sigma, p.alpha)
    xs = [f32(p.x0)]
    for _ in range(n + count - 1):
        xs.append(f32(F(xs[-1])))
    return xs[n:]


def compare(P, xs_dev, method):
    torch = torch_cuda()
    out_ref = torch.empty_like(xs_dev[0])
    out_st = torch.full_like(xs_dev[0], float("nan"))
    st_ref, g_ref = P.ve_extrapolate(xs_dev, out_ref)
    st, g = red.ve_extrapolate_static(xs_dev, out_st, method)
    torch.cuda.synchronize()
    assert st == st_ref
    if g_ref is not None:
        np.testing.assert_allclose(g, g_ref, rtol=GAMMA_RTOL, atol=1e-12)
    assert float((out_st - out_ref).abs().max()) <= 1e-4


@pytest.mark.parametrize("method", ["mpe", "rre", "svdmpe"])
def test_static_matches_problem_entry_point_two_calls(method):
    p = synth.make_deblur(5, 64, 64, synth.uniform_psf(9), 2 ** 0.5)
    P = red.Problem(red.config_for(p, ve=method, ve_k=5), to_dev(p.y))
    hist = fp_history(p, 2, 8)
    first = [to_dev(x) for x in hist[:6]]      # x_2 .. x_7 (kappa = 4)
    second = [to_dev(x) for x in hist[2:8]]    # x_4 .. x_9: a second call right after
    compare(P, first, method)
    compare(P, second, method)


def test_static_unaligned_ragged_and_many_chunks():
    """n = 81 x 54 (not a multiple of 4) at a 4-byte offset (scalar paths), and a vector
    of 1152 chunks of 2048 (more chunks than Gram CTAs: each CTA sums several chunks)."""
    torch = torch_cuda()
    p = synth.make_deblur(7, 81, 54, synth.uniform_psf(5), 2 ** 0.5)
    P = red.Problem(red.config_for(p, ve="rre", ve_k=4), to_dev(p.y))
    hist = fp_history(p, 1, 5)
    n = 81 * 54
    big = torch.empty(5 * (n + 1) + 1, device="cuda")
    xs = []
    for i, x in enumerate(hist):
        v = big[1 + i * (n + 1): 1 + i * (n + 1) + n].view(81, 54)
        v.copy_(to_dev(x))
        xs.append(v)
    out_ref = torch.empty((81, 54), device="cuda")
    st_ref, g_ref = P.ve_extrapolate(xs, out_ref)
    flat = [x.reshape(-1) for x in xs]
    out = torch.empty(n + 1, device="cuda")[1:]
    st, g = red.ve_extrapolate_static(flat, out, "rre")
    assert st == st_ref == red.RED_OK
    np.testing.assert_allclose(g, g_ref, rtol=GAMMA_RTOL, atol=1e-12)
    assert float((out.view(81, 54) - out_ref).abs().max()) <= 1e-4

    # 1152 chunks of 2048: a linear map with 3 distinct eigenvalues; kappa = 3 (x_0 .. x_4,
    # four differences) reaches its fixed point (Eqs. (13)-(16))
    H, W = 1152, 2048
    q = synth.make_deblur(3, H, W, synth.uniform_psf(3), 2 ** 0.5)
    Q = red.Problem(red.config_for(q, ve="rre", ve_k=4), to_dev(q.y))
    gen = torch.Generator(device="cuda").manual_seed(3)
    m = H * W
    lam = torch.tensor([0.9, -0.4, 0.5], device="cuda").repeat_interleave(m // 3 + 1)[:m]
    b = torch.rand(m, device="cuda", generator=gen) * 10 - 5
    vs = [torch.rand(m, device="cuda", generator=gen) * 100]
    for _ in range(4):
        vs.append(lam * vs[-1] + b)
    out_ref = torch.empty((H, W), device="cuda")
    st_ref, g_ref = Q.ve_extrapolate([v.view(H, W) for v in vs], out_ref)
    out = torch.empty(m, device="cuda")
    st, g = red.ve_extrapolate_static(vs, out, "rre")
    assert st == st_ref == red.RED_OK
    np.testing.assert_allclose(g, g_ref, rtol=GAMMA_RTOL, atol=1e-12)
    assert float((out.view(H, W) - out_ref).abs().max()) <= 1e-4
    fixed = b.double() / (1 - lam.double())
    assert float((out.double() - fixed).abs().max()) <= 1e-3 * float(fixed.abs().max())


def test_static_breakdown_and_no_device_allocation():
    torch = torch_cuda()
    v = torch.arange(64 * 64, dtype=torch.float32, device="cuda") / 100
    drift = [v * 0, v * 1, v * 2]                # pure drift: MPE's sum c = 0
    out = torch.empty_like(v)
    red.ve_extrapolate_static(drift, out, "mpe")  # the first call on the device did setup
    assert torch.equal(out, drift[-1])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    results = [red.ve_extrapolate_static(drift, out, "mpe") for _ in range(3)]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert all(st == red.RED_EVE_BREAKDOWN and g is None for st, g in results)
    assert torch.equal(out, drift[-1])


def test_static_rejects_sizes_beyond_limit():
    torch = torch_cuda()
    v = torch.zeros(16, device="cuda")
    L = red.lib()
    arr = (ctypes.c_void_p * 3)(*[v.data_ptr()] * 3)
    gam = (ctypes.c_double * 16)()
    st = L.red_ve_extrapolate_static(arr, 3, 2 ** 31, 2, ctypes.c_void_p(v.data_ptr()), gam, None)
    assert st == red.RED_EINVAL
    assert b"exceeds the limit" in L.red_last_error()
    arr14 = (ctypes.c_void_p * 14)(*[v.data_ptr()] * 14)
    st = L.red_ve_extrapolate_static(arr14, 14, 16, 2, ctypes.c_void_p(v.data_ptr()), gam, None)
    assert st == red.RED_EINVAL
    st = L.red_ve_extrapolate_static(arr, 3, 16, 0, ctypes.c_void_p(v.data_ptr()), gam, None)
    assert st == red.RED_EINVAL
