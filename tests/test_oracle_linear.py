"""Pins for the oracle's linear algebra: the circulant blur H, decimation S, the
Fourier-domain inverse of Eq. (7) (footnote: block-circulant H) and the CG solve used
for super-resolution. Every check builds the operator as an explicit dense matrix from
the PSF taps (no FFT) or uses the problem's closed-form optimality condition."""
import math

import numpy as np
import pytest

from oracle import operators as ops
from oracle import fp
from paper_1805_02158_gb300 import synth


def dense_blur_matrix(psf, h, w):
    """Circular convolution as an explicit (h*w) x (h*w) matrix, built tap by tap."""
    k1, k2 = psf.shape
    c1, c2 = (k1 - 1) // 2, (k2 - 1) // 2
    M = np.zeros((h * w, h * w))
    for i in range(h):
        for j in range(w):
            for a in range(k1):
                for b in range(k2):
                    si, sj = (i - (a - c1)) % h, (j - (b - c2)) % w
                    M[i * w + j, si * w + sj] += psf[a, b]
    return M


def dense_decimation(h, w, s):
    lh, lw = h // s, w // s
    S = np.zeros((lh * lw, h * w))
    for i in range(lh):
        for j in range(lw):
            S[i * lw + j, (s * i) * w + s * j] = 1.0
    return S


@pytest.mark.parametrize("shape,psf", [((8, 8), synth.uniform_psf(3)),
                                       ((6, 10), synth.gaussian_psf(5, 1.2)),
                                       ((9, 12), synth.gaussian_psf(7, 1.6))])
def test_blur_and_adjoint_match_dense(shape, psf):
    h, w = shape
    rng = np.random.default_rng(0)
    x = rng.standard_normal(shape)
    M = dense_blur_matrix(psf, h, w)
    otf = ops.psf_otf(psf, shape)
    np.testing.assert_allclose(ops.blur(x, otf).ravel(), M @ x.ravel(), atol=1e-12)
    np.testing.assert_allclose(ops.blur_adjoint(x, otf).ravel(), M.T @ x.ravel(), atol=1e-12)
    # the generator's tap-by-tap blur is the same operator
    np.testing.assert_allclose(synth.circular_blur_direct(x, psf), ops.blur(x, otf), atol=1e-12)


def test_asymmetric_psf_orientation():
    psf = np.zeros((3, 3))
    psf[0, 2] = 1.0  # shift kernel: offset (-1, +1) from the centre
    x = np.random.default_rng(1).standard_normal((5, 7))
    otf = ops.psf_otf(psf, x.shape)
    M = dense_blur_matrix(psf, 5, 7)
    np.testing.assert_allclose(ops.blur(x, otf).ravel(), M @ x.ravel(), atol=1e-12)
    np.testing.assert_allclose(ops.blur(x, otf), np.roll(x, (-1, 1), axis=(0, 1)), atol=1e-12)


@pytest.mark.parametrize("shape,psf,sigma,alpha", [((8, 8), synth.uniform_psf(3), math.sqrt(2), 0.02),
                                                   ((6, 10), synth.gaussian_psf(5, 1.6), 2.0, 0.3)])
def test_deblur_solve_equals_dense_solve(shape, psf, sigma, alpha):
    h, w = shape
    rng = np.random.default_rng(2)
    y = rng.uniform(0, 255, shape)
    f = rng.uniform(0, 255, shape)
    M = dense_blur_matrix(psf, h, w)
    A = M.T @ M / sigma ** 2 + alpha * np.eye(h * w)
    b = M.T @ y.ravel() / sigma ** 2 + alpha * f.ravel()
    x_dense = np.linalg.solve(A, b)
    x = fp.deblur_solve(f, y, ops.psf_otf(psf, shape), sigma, alpha)
    np.testing.assert_allclose(x.ravel(), x_dense, rtol=1e-10, atol=1e-9)


def test_deblur_solve_satisfies_normal_equations_64():
    p = synth.deblur_small(0)
    rng = np.random.default_rng(3)
    f = rng.uniform(0, 255, p.y.shape)
    x = fp.deblur_solve(f, p.y, ops.psf_otf(p.psf, p.y.shape), p.sigma, p.alpha)
    hx = synth.circular_blur_direct(x, p.psf)
    hthx = synth.circular_blur_direct(hx, p.psf[::-1, ::-1])
    hty = synth.circular_blur_direct(p.y, p.psf[::-1, ::-1])
    res = hthx / p.sigma ** 2 + p.alpha * x - (hty / p.sigma ** 2 + p.alpha * f)
    assert np.abs(res).max() < 1e-9 * np.abs(hty / p.sigma ** 2).max()


def test_sr_adjoint_identity():
    rng = np.random.default_rng(4)
    psf = synth.gaussian_psf(7, 1.6)
    shape = (13, 11)
    otf = ops.psf_otf(psf, shape)
    p = rng.standard_normal(shape)
    q = rng.standard_normal((13 // 3, 11 // 3))
    lhs = float(np.vdot(ops.forward(p, otf, 3), q))
    rhs = float(np.vdot(p, ops.adjoint(q, otf, 3, shape)))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_sr_operator_matches_dense_and_cg_reaches_dense_solve():
    h = w = 12
    s = 3
    sigma, alpha = 5.0, 0.02
    psf = synth.gaussian_psf(7, 1.6)
    otf = ops.psf_otf(psf, (h, w))
    B = dense_blur_matrix(psf, h, w)
    S = dense_decimation(h, w, s)
    A = (S @ B).T @ (S @ B) / sigma ** 2 + alpha * np.eye(h * w)
    rng = np.random.default_rng(5)
    v = rng.standard_normal((h, w))
    np.testing.assert_allclose(fp.sr_normal_apply(v, otf, s, sigma, alpha).ravel(), A @ v.ravel(),
                               atol=1e-12)
    y = rng.uniform(0, 255, (h // s, w // s))
    f = rng.uniform(0, 255, (h, w))
    b = fp.sr_rhs(f, y, otf, s, sigma, alpha)
    np.testing.assert_allclose(b.ravel(), (S @ B).T @ y.ravel() / sigma ** 2 + alpha * f.ravel(),
                               atol=1e-10)
    x_dense = np.linalg.solve(A, b.ravel())
    x_cg = fp.conjugate_gradient(lambda t: fp.sr_normal_apply(t, otf, s, sigma, alpha), b,
                                 np.zeros((h, w)), 400)
    np.testing.assert_allclose(x_cg.ravel(), x_dense, rtol=1e-9, atol=1e-7)


def test_cg_energy_error_decreases():
    rng = np.random.default_rng(6)
    n = 40
    G = rng.standard_normal((n, n))
    A = G @ G.T / n + np.eye(n)
    b = rng.standard_normal(n)
    xs = np.linalg.solve(A, b)
    errs = []
    for it in range(0, 25):
        x = fp.conjugate_gradient(lambda v: A @ v, b, np.zeros(n), it)
        e = x - xs
        errs.append(float(e @ A @ e))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(len(errs) - 1))
    assert errs[-1] < 1e-6 * errs[0]


def test_deblur_solve_with_an_asymmetric_psf_equals_dense_solve():
    """A non-symmetric PSF has a complex spectrum, so the conjugate in H^T of Eq. (7)
    matters (the paper's PSFs are symmetric and real-spectrum; the solve is defined for any
    circulant H)."""
    rng = np.random.default_rng(7)
    psf = rng.uniform(0, 1, (3, 5))
    psf /= psf.sum()
    h, w, sigma, alpha = 6, 10, 1.5, 0.1
    y = rng.uniform(0, 255, (h, w))
    f = rng.uniform(0, 255, (h, w))
    M = dense_blur_matrix(psf, h, w)
    A = M.T @ M / sigma ** 2 + alpha * np.eye(h * w)
    x_dense = np.linalg.solve(A, M.T @ y.ravel() / sigma ** 2 + alpha * f.ravel())
    x = fp.deblur_solve(f, y, ops.psf_otf(psf, (h, w)), sigma, alpha)
    np.testing.assert_allclose(x.ravel(), x_dense, rtol=1e-10, atol=1e-9)


def test_sr_fp_step_warm_starts_cg_at_the_current_iterate():
    """Reading: CG starts from x_k. With 0 iterations the SR FP step returns x_k; with one
    it is the exact line-search step from x_k along r = b - A x_k, x_k + (r^T r / r^T A r) r,
    written here with the dense A and b."""
    h = w = 12
    s, sigma, alpha = 3, 5.0, 0.02
    psf = synth.gaussian_psf(7, 1.6)
    B = dense_blur_matrix(psf, h, w)
    S = dense_decimation(h, w, s)
    A = (S @ B).T @ (S @ B) / sigma ** 2 + alpha * np.eye(h * w)
    rng = np.random.default_rng(8)
    y = rng.uniform(0, 255, (h // s, w // s))
    xk = rng.uniform(0, 255, (h, w))
    F0 = fp.FPOperator(y, psf, (h, w), s, sigma, alpha, cg_iters=0)
    np.testing.assert_array_equal(F0(xk), xk)
    F1 = fp.FPOperator(y, psf, (h, w), s, sigma, alpha, cg_iters=1)
    x1, f = F1.step_with_f(xk)
    b = (S @ B).T @ y.ravel() / sigma ** 2 + alpha * f.ravel()
    r = b - A @ xk.ravel()
    expect = xk.ravel() + (r @ r) / (r @ A @ r) * r
    np.testing.assert_allclose(x1.ravel(), expect, rtol=1e-10, atol=1e-8)
    # the module-level step takes the same path
    np.testing.assert_allclose(fp.sr_fp_step(xk, y, ops.psf_otf(psf, (h, w)), s, sigma, alpha,
                                             cg_iters=1), x1, rtol=1e-13, atol=1e-10)
