"""Seeded synthetic inputs for RED deblurring and super-resolution problems.

The paper's test images (Sec. IV-A, Table I; Sec. IV-B, Table II) are not available,
so every problem here is drawn from a seed: a piecewise-smooth "ellipses + ramps +
texture" image in [0, 255], a point-spread function, white Gaussian noise, and the
observation y = H x_true + e of Eq. (1) (H = circular blur, or circular blur followed
by decimation for super-resolution).

This module holds none of the solver's arithmetic: it never denoises, never inverts H
and never extrapolates. It only draws inputs, so both the FP64 oracle tests and the GPU
harness can take bit-identical inputs from it. The observation is formed with a direct
(tap-by-tap) circular convolution, which is independent of the FFT-based operators used
by the oracle and by the CUDA path.

Random numbers come from SplitMix64 used as a counter-based generator
(output_i = mix(key + (i + 1) * 0x9E3779B97F4A7C15)), uniforms as the top 53 bits
scaled by 2^-53, normals by the Box-Muller cosine branch.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream tags: each seed owns independent streams for image shape, texture and noise.
TAG_IMAGE = 1
TAG_TEXTURE = 2
TAG_NOISE = 3
TAG_PROBLEM = 4
TAG_ARRIVALS = 5


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(key: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 outputs for the given counters under a 64-bit key (wrapping uint64)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (c + np.uint64(1)) * _GOLDEN
    return _mix(z)


class Stream:
    """A counter-based random stream identified by (seed, tag)."""

    def __init__(self, seed: int, tag: int):
        k = np.array([(int(seed) * 1315423911 + int(tag) * 2654435761) & 0xFFFFFFFFFFFFFFFF],
                     dtype=np.uint64)
        self.key = int(_mix(k)[0])
        self.pos = 0

    def uniform(self, n: int) -> np.ndarray:
        z = splitmix64(self.key, np.arange(self.pos, self.pos + n, dtype=np.uint64))
        self.pos += n
        return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def uniform1(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return float(lo + (hi - lo) * self.uniform(1)[0])

    def normal(self, n: int) -> np.ndarray:
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)

    def choice(self, options):
        i = min(int(self.uniform(1)[0] * len(options)), len(options) - 1)
        return options[i]


def ellipse_image(seed: int, height: int, width: int, n_ellipses: int = 12,
                  texture_sigma: float = 5.0) -> np.ndarray:
    """Piecewise-smooth ground truth in [0, 255]: constant background, n_ellipses
    ellipses painted in order, each with a linear intensity ramp, plus N(0, 5^2)
    texture, clipped to [0, 255]. Returns float64 [height, width]."""
    s = Stream(seed, TAG_IMAGE)
    side = float(min(height, width))
    img = np.full((height, width), s.uniform1(0.0, 255.0))
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    for _ in range(n_ellipses):
        cx = s.uniform1(0.0, width)
        cy = s.uniform1(0.0, height)
        ra = s.uniform1(side / 16.0, side / 3.0)
        rb = s.uniform1(side / 16.0, side / 3.0)
        th = s.uniform1(0.0, math.pi)
        a = s.uniform1(0.0, 255.0)
        gx = s.uniform1(-1.0, 1.0) * 255.0 / width
        gy = s.uniform1(-1.0, 1.0) * 255.0 / height
        dx = xx - cx
        dy = yy - cy
        c, sn = math.cos(th), math.sin(th)
        u = (dx * c + dy * sn) / ra
        v = (-dx * sn + dy * c) / rb
        inside = u * u + v * v <= 1.0
        img = np.where(inside, a + gx * dx + gy * dy, img)
    t = Stream(seed, TAG_TEXTURE)
    img = img + texture_sigma * t.normal(height * width).reshape(height, width)
    return np.clip(img, 0.0, 255.0)


def uniform_psf(k: int) -> np.ndarray:
    return np.full((k, k), 1.0 / (k * k))


def gaussian_psf(k: int, s: float) -> np.ndarray:
    r = (k - 1) / 2.0
    a = np.arange(k, dtype=np.float64) - r
    g = np.exp(-(a[:, None] ** 2 + a[None, :] ** 2) / (2.0 * s * s))
    return g / g.sum()


def circular_blur_direct(x: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """Tap-by-tap circular convolution with the PSF centred at ((K1-1)/2, (K2-1)/2)."""
    k1, k2 = psf.shape
    c1, c2 = (k1 - 1) // 2, (k2 - 1) // 2
    out = np.zeros_like(x, dtype=np.float64)
    for a in range(k1):
        for b in range(k2):
            out += psf[a, b] * np.roll(x, shift=(a - c1, b - c2), axis=(0, 1))
    return out


def gaussian_taps(k: int, s: float) -> np.ndarray:
    """1-D factor of gaussian_psf: gaussian_psf(k, s) = outer(t, t) with t = these taps."""
    r = (k - 1) / 2.0
    a = np.arange(k, dtype=np.float64) - r
    g = np.exp(-(a ** 2) / (2.0 * s * s))
    return g / g.sum()


def circular_blur_separable(x: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Circular convolution with the PSF outer(u, v) (centre ((K1-1)/2, (K2-1)/2)), as a
    column pass then a row pass of taps: the same result as circular_blur_direct with that
    PSF up to rounding, with K1 + K2 instead of K1 K2 passes (used for large images)."""
    c1, c2 = (len(u) - 1) // 2, (len(v) - 1) // 2
    t = np.zeros_like(x, dtype=np.float64)
    for a in range(len(u)):
        t += u[a] * np.roll(x, shift=a - c1, axis=0)
    out = np.zeros_like(x, dtype=np.float64)
    for b in range(len(v)):
        out += v[b] * np.roll(t, shift=b - c2, axis=1)
    return out


def lr_shape(height: int, width: int, scale: int):
    return height // scale, width // scale


@dataclass
class Problem:
    """One synthetic RED problem. Arrays are float64; `y32`/`x0_32` are the float32
    roundings handed to the GPU, and the oracle is fed the same float32 values."""
    seed: int
    task: str                 # "deblur" or "sr"
    height: int
    width: int
    scale: int
    psf: np.ndarray
    sigma: float
    alpha: float
    x_true: np.ndarray
    y: np.ndarray
    x0: np.ndarray
    nlm_patch: int = 5
    nlm_search: int = 11
    nlm_h: float = 10.0
    meta: dict = field(default_factory=dict)

    @property
    def y32(self) -> np.ndarray:
        return self.y.astype(np.float32)

    @property
    def x0_32(self) -> np.ndarray:
        return self.x0.astype(np.float32)

    @property
    def psf32(self) -> np.ndarray:
        return self.psf.astype(np.float32)


def upsample_replicate(z: np.ndarray, scale: int, height: int, width: int) -> np.ndarray:
    """Pixel replication of an LR image by scale x scale blocks, edge-extended to
    (height, width). Used as the super-resolution initial guess."""
    up = np.repeat(np.repeat(z, scale, axis=0), scale, axis=1)
    ri = np.minimum(np.arange(height), up.shape[0] - 1)
    ci = np.minimum(np.arange(width), up.shape[1] - 1)
    return up[np.ix_(ri, ci)]


def make_deblur(seed: int, height: int, width: int, psf: np.ndarray, sigma: float,
                alpha: float = 0.02, blur=None) -> Problem:
    """blur: optional callable x -> H x (default: circular_blur_direct with psf)."""
    x = ellipse_image(seed, height, width)
    n = Stream(seed, TAG_NOISE).normal(height * width).reshape(height, width)
    hx = blur(x) if blur is not None else circular_blur_direct(x, psf)
    y = hx + sigma * n
    return Problem(seed=seed, task="deblur", height=height, width=width, scale=1, psf=psf,
                   sigma=sigma, alpha=alpha, x_true=x, y=y, x0=y.copy())


def make_sr(seed: int, height: int, width: int, psf: np.ndarray, scale: int, sigma: float,
            alpha: float = 0.02, blur=None) -> Problem:
    x = ellipse_image(seed, height, width)
    h, w = lr_shape(height, width, scale)
    n = Stream(seed, TAG_NOISE).normal(h * w).reshape(h, w)
    hx = blur(x) if blur is not None else circular_blur_direct(x, psf)
    y = hx[: scale * h: scale, : scale * w: scale] + sigma * n
    x0 = upsample_replicate(y, scale, height, width)
    return Problem(seed=seed, task="sr", height=height, width=width, scale=scale, psf=psf,
                   sigma=sigma, alpha=alpha, x_true=x, y=y, x0=x0)


# ---------------------------------------------------------------------------------------
# Workloads. Each mirrors one of the paper's experiment families with synthetic images.
# ---------------------------------------------------------------------------------------

def deblur_small(seed: int = 0, side: int = 64) -> Problem:
    """64x64 deblurring, 9x9 uniform PSF, noise sigma sqrt(2) (Sec. IV-A setting)."""
    return make_deblur(seed, side, side, uniform_psf(9), math.sqrt(2.0))


def deblur_gauss256(seed: int, side: int = 256) -> Problem:
    """256x256 deblurring, 25x25 Gaussian PSF with std 1.6, noise sigma sqrt(2)."""
    return make_deblur(seed, side, side, gaussian_psf(25, 1.6), math.sqrt(2.0))


def sr_x3(seed: int, side: int = 256) -> Problem:
    """x3 super-resolution: 7x7 Gaussian PSF std 1.6, decimation by 3, noise sigma 5
    (Sec. IV-B setting)."""
    return make_sr(seed, side, side, gaussian_psf(7, 1.6), 3, 5.0)


BATCH_SIDES = (128, 192, 256, 384, 512)


def batched_uneven(seed: int) -> Problem:
    """One problem of the uneven batch: side drawn from {128,192,256,384,512}; PSF
    uniform 9x9 with probability 1/2, else Gaussian with std U[1,2] and size
    2*ceil(3 std)+1; noise sigma U[1,5]."""
    s = Stream(seed, TAG_PROBLEM)
    side = s.choice(BATCH_SIDES)
    if s.uniform1() < 0.5:
        psf = uniform_psf(9)
    else:
        sd = s.uniform1(1.0, 2.0)
        psf = gaussian_psf(2 * math.ceil(3 * sd) + 1, sd)
    sigma = s.uniform1(1.0, 5.0)
    p = make_deblur(seed, side, side, psf, sigma)
    return p


SERVE_SIDES = (128, 192, 256, 384, 512, 768, 1024)


def serving_request(seed: int) -> Problem:
    """One request of the serving stream: 70% deblurring (Gaussian 25x25 std 1.6,
    sigma sqrt 2), 30% x3 super-resolution (Sec. IV-B physics); side drawn from
    {128,...,1024}. The Gaussian blur is applied as two 1-D passes (large sides)."""
    s = Stream(seed, TAG_PROBLEM)
    side = s.choice(SERVE_SIDES)
    if s.uniform1() < 0.7:
        t = gaussian_taps(25, 1.6)
        return make_deblur(seed, side, side, gaussian_psf(25, 1.6), math.sqrt(2.0),
                           blur=lambda x: circular_blur_separable(x, t, t))
    t = gaussian_taps(7, 1.6)
    return make_sr(seed, side, side, gaussian_psf(7, 1.6), 3, 5.0,
                   blur=lambda x: circular_blur_separable(x, t, t))


def poisson_arrivals(rate_hz: float, n: int, seed: int = 0) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    u = Stream(seed, TAG_ARRIVALS).uniform(n)
    gaps = -np.log1p(-u) / rate_hz
    return np.cumsum(gaps)
