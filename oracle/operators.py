"""Degradation operators of Eq. (1) in FP64.

H is a circular (block-circulant) blur for deblurring, and S B (blur, then keep every
scale-th sample starting at index 0) for super-resolution. The blur is applied in the
Fourier domain, where a block-circulant operator is diagonal (footnote to Eq. (7)):
K_hat = FFT2 of the PSF zero-padded to the image size and circularly shifted so that
its centre ((K1-1)/2, (K2-1)/2) sits at the origin.
"""
from __future__ import annotations

import numpy as np


def psf_otf(psf: np.ndarray, shape) -> np.ndarray:
    h, w = shape
    k1, k2 = psf.shape
    pad = np.zeros((h, w), dtype=np.float64)
    pad[:k1, :k2] = psf
    pad = np.roll(pad, shift=(-((k1 - 1) // 2), -((k2 - 1) // 2)), axis=(0, 1))
    return np.fft.fft2(pad)


def blur(x: np.ndarray, otf: np.ndarray) -> np.ndarray:
    return np.real(np.fft.ifft2(otf * np.fft.fft2(x)))


def blur_adjoint(x: np.ndarray, otf: np.ndarray) -> np.ndarray:
    return np.real(np.fft.ifft2(np.conj(otf) * np.fft.fft2(x)))


def decimate(x: np.ndarray, scale: int) -> np.ndarray:
    h, w = x.shape[0] // scale, x.shape[1] // scale
    return x[: scale * h: scale, : scale * w: scale]


def decimate_adjoint(z: np.ndarray, scale: int, shape) -> np.ndarray:
    out = np.zeros(shape, dtype=np.float64)
    h, w = z.shape
    out[: scale * h: scale, : scale * w: scale] = z
    return out


def forward(x: np.ndarray, otf: np.ndarray, scale: int) -> np.ndarray:
    """H x of Eq. (1)."""
    bx = blur(x, otf)
    return bx if scale == 1 else decimate(bx, scale)


def adjoint(z: np.ndarray, otf: np.ndarray, scale: int, shape) -> np.ndarray:
    """H^T z."""
    if scale != 1:
        z = decimate_adjoint(z, scale, shape)
    return blur_adjoint(z, otf)
