"""One fixed-point (FP) step of RED, Eq. (7) (Sec. II-B), in FP64:

    x_{k+1} = [H^T H / sigma^2 + alpha I]^{-1} [H^T y / sigma^2 + alpha f(x_k)]

The inverse is applied in the Fourier domain for a block-circulant H (deblurring) and by
an iterative method otherwise (footnote to Eq. (7)); for super-resolution that method is
conjugate gradients on the normal equations with a fixed iteration count, warm-started at
x_k, with no preconditioner and the residual formed afresh from b - A x_k.
"""
from __future__ import annotations

import numpy as np

from . import operators as ops
from .nlm import nlm


def deblur_solve(f: np.ndarray, y: np.ndarray, otf: np.ndarray, sigma: float,
                 alpha: float) -> np.ndarray:
    """The linear part of Eq. (7) for a circulant H: the matrix is diagonal in Fourier
    space with entries |K_hat|^2 / sigma^2 + alpha."""
    rhs_hat = np.conj(otf) * np.fft.fft2(y) / sigma ** 2 + alpha * np.fft.fft2(f)
    diag = np.abs(otf) ** 2 / sigma ** 2 + alpha
    return np.real(np.fft.ifft2(rhs_hat / diag))


def deblur_fp_step(x: np.ndarray, y: np.ndarray, otf: np.ndarray, sigma: float,
                   alpha: float, denoise=nlm) -> np.ndarray:
    return deblur_solve(denoise(x), y, otf, sigma, alpha)


def sr_normal_apply(p: np.ndarray, otf: np.ndarray, scale: int, sigma: float,
                    alpha: float) -> np.ndarray:
    """(B^T S^T S B / sigma^2 + alpha I) p for H = S B."""
    hp = ops.forward(p, otf, scale)
    return ops.adjoint(hp, otf, scale, p.shape) / sigma ** 2 + alpha * p


def conjugate_gradient(apply_a, b: np.ndarray, x0: np.ndarray, iters: int) -> np.ndarray:
    """Textbook CG (Hestenes-Stiefel) for a symmetric positive definite operator, run
    for exactly `iters` iterations (stopping early only once the residual or p^T A p has
    underflowed to 0)."""
    x = x0.copy()
    r = b - apply_a(x)
    p = r.copy()
    rr = float(np.vdot(r, r))
    for _ in range(iters):
        if rr == 0.0:
            break
        ap = apply_a(p)
        pap = float(np.vdot(p, ap))
        if pap <= 0.0:   # only after full convergence (underflow); the operator is SPD
            break
        a = rr / pap
        x = x + a * p
        r = r - a * ap
        rr_new = float(np.vdot(r, r))
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    return x


def sr_rhs(f: np.ndarray, y: np.ndarray, otf: np.ndarray, scale: int, sigma: float,
           alpha: float) -> np.ndarray:
    return ops.adjoint(y, otf, scale, f.shape) / sigma ** 2 + alpha * f


def sr_fp_step(x: np.ndarray, y: np.ndarray, otf: np.ndarray, scale: int, sigma: float,
               alpha: float, cg_iters: int = 20, denoise=nlm) -> np.ndarray:
    f = denoise(x)
    b = sr_rhs(f, y, otf, scale, sigma, alpha)
    return conjugate_gradient(lambda v: sr_normal_apply(v, otf, scale, sigma, alpha),
                              b, x, cg_iters)


class FPOperator:
    """The FP map x -> F(x) of Eq. (17) for one problem, with the problem's physics."""

    def __init__(self, y, psf, shape, scale, sigma, alpha, patch=5, search=11, h=10.0,
                 cg_iters=20):
        self.y = np.asarray(y, dtype=np.float64)
        self.shape = tuple(shape)
        self.scale = int(scale)
        self.sigma = float(sigma)
        self.alpha = float(alpha)
        self.otf = ops.psf_otf(np.asarray(psf, dtype=np.float64), self.shape)
        self.patch, self.search, self.h = patch, search, h
        self.cg_iters = cg_iters

    def denoise(self, x):
        return nlm(x, self.patch, self.search, self.h)

    def solve_linear(self, f, x_warm):
        if self.scale == 1:
            return deblur_solve(f, self.y, self.otf, self.sigma, self.alpha)
        b = sr_rhs(f, self.y, self.otf, self.scale, self.sigma, self.alpha)
        return conjugate_gradient(
            lambda v: sr_normal_apply(v, self.otf, self.scale, self.sigma, self.alpha),
            b, x_warm, self.cg_iters)

    def __call__(self, x):
        return self.solve_linear(self.denoise(x), x)

    def step_with_f(self, x):
        """Returns (F(x), f(x)) so callers can reuse f(x) for the objective."""
        f = self.denoise(x)
        return self.solve_linear(f, x), f
