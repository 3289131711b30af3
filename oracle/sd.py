"""The steepest-descent (SD) baseline of SD-MPE (Sec. IV-A, Sec. IV-B) in FP64.

TEST INFRASTRUCTURE ONLY (see the package header): nothing on the product path imports it.

One SD step moves against the gradient of the RED objective, Eq. (5):

    x_{k+1} = x_k - mu * ( H^T (H x_k - y) / sigma^2 + alpha (x_k - f(x_k)) )

with a fixed step size mu. Each step costs one denoiser call, like an FP step of Eq. (7).
SD-MPE is Algorithm 3 with this map as the baseline algorithm in place of FP (the paper
uses m = 0, kappa = 8 for deblurring and m = 1, kappa = 10 for super-resolution); the
cycling driver `red.solve` takes any baseline map, so SD-MPE is `red.solve(SDOperator(..),
x0, "mpe", m, kappa, ...)`.

Reading where the paper is silent: the step size. The paper picks a fixed mu by hand
(a line search would cost extra denoiser calls) and does not print it. The default here is
mu = 1 / (max |K_hat|^2 / sigma^2 + alpha), the reciprocal of the largest eigenvalue of
H^T H / sigma^2 + alpha I, i.e. of the objective's Hessian with the denoiser's Jacobian
taken as 0. For super-resolution H^T H = B^T S^T S B, whose largest eigenvalue is at most
max |K_hat|^2 (S^T S is a projection), so the same mu is a safe step there. Any mu may be
passed instead.
"""
from __future__ import annotations

import numpy as np

from . import operators as ops
from .nlm import nlm
from .red import gradient


def default_step(otf: np.ndarray, sigma: float, alpha: float) -> float:
    """mu = 1 / (max |K_hat|^2 / sigma^2 + alpha)."""
    return 1.0 / (float(np.max(np.abs(otf) ** 2)) / sigma ** 2 + alpha)


class SDOperator:
    """The SD map x -> x - mu grad E(x) for one problem (same physics as fp.FPOperator).
    `denoise` replaces the NLM denoiser (used by the pins with a linear denoiser)."""

    def __init__(self, y, psf, shape, scale, sigma, alpha, mu=None, patch=5, search=11,
                 h=10.0, denoise=None):
        self.y = np.asarray(y, dtype=np.float64)
        self.shape = tuple(shape)
        self.scale = int(scale)
        self.sigma = float(sigma)
        self.alpha = float(alpha)
        self.otf = ops.psf_otf(np.asarray(psf, dtype=np.float64), self.shape)
        self.mu = default_step(self.otf, self.sigma, self.alpha) if mu is None else float(mu)
        self.patch, self.search, self.h = patch, search, h
        self._denoise = denoise

    def denoise(self, x):
        if self._denoise is not None:
            return self._denoise(x)
        return nlm(x, self.patch, self.search, self.h)

    def step_with_f(self, x):
        """Returns (SD step from x, f(x))."""
        f = self.denoise(x)
        g = gradient(x, f, self.y, self.otf, self.scale, self.sigma, self.alpha)
        return x - self.mu * g, f

    def __call__(self, x):
        return self.step_with_f(x)[0]
