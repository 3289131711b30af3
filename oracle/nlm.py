"""The denoiser f(x) of Eq. (3) (Sec. II-B): pixelwise non-local means, FP64.

The paper uses TNRD as the denoising engine (Sec. IV) and treats f only as an abstract
differentiable denoiser (Sec. II-B). Here f is classic pixelwise non-local means with
these readings:

  f(p) = sum_{d in S} w(p, d) xp(p + d) / sum_{d in S} w(p, d)
  w(p, d) = exp( -(1 / (P^2 h^2)) * sum_{t in T} (xp(p + t) - xp(p + d + t))^2 )

where S = [-s, s]^2 is the search window (s = search // 2, 11x11 by default),
T = [-r, r]^2 the patch (r = patch // 2, 5x5 by default), P = patch, h the filtering
parameter (10 on the [0, 255] scale), the self candidate d = 0 is included with weight 1,
and xp is x extended beyond the image by half-sample symmetric reflection (index -1 -> 0,
n -> n-1), applied to both the search window and the patches.
"""
from __future__ import annotations

import numpy as np


def mirror_index(i, n: int):
    """Half-sample symmetric reflection of integer index i into [0, n) (period 2n)."""
    p = 2 * n
    i = np.mod(i, p)
    return np.where(i < n, i, p - 1 - i)


def pad_symmetric(x: np.ndarray, r: int) -> np.ndarray:
    h, w = x.shape
    rows = mirror_index(np.arange(-r, h + r), h)
    cols = mirror_index(np.arange(-r, w + r), w)
    return x[np.ix_(rows, cols)]


def nlm(x: np.ndarray, patch: int = 5, search: int = 11, h: float = 10.0) -> np.ndarray:
    """Direct-form non-local means over the whole image (vectorised over pixels; each
    patch distance is the plain 25-term sum of squared differences)."""
    x = np.asarray(x, dtype=np.float64)
    hh, ww = x.shape
    pr, sr = patch // 2, search // 2
    rad = pr + sr
    xp = pad_symmetric(x, rad)
    scale = 1.0 / (patch * patch * h * h)
    num = np.zeros_like(x)
    den = np.zeros_like(x)
    for dy in range(-sr, sr + 1):
        for dx in range(-sr, sr + 1):
            dist = np.zeros_like(x)
            for ty in range(-pr, pr + 1):
                for tx in range(-pr, pr + 1):
                    a = xp[rad + ty: rad + ty + hh, rad + tx: rad + tx + ww]
                    b = xp[rad + dy + ty: rad + dy + ty + hh, rad + dx + tx: rad + dx + tx + ww]
                    dist += (a - b) ** 2
            w = np.exp(-dist * scale)
            num += w * xp[rad + dy: rad + dy + hh, rad + dx: rad + dx + ww]
            den += w
    return num / den


def nlm_pixel(x: np.ndarray, i: int, j: int, patch: int = 5, search: int = 11,
              h: float = 10.0) -> float:
    """f at one pixel (i, j), written out from the definition with scalar loops. Used for
    sampled checks at sizes where the whole-image oracle would be slow."""
    hh, ww = x.shape
    pr, sr = patch // 2, search // 2

    def px(a, b):
        return float(x[int(mirror_index(a, hh)), int(mirror_index(b, ww))])

    num = 0.0
    den = 0.0
    for dy in range(-sr, sr + 1):
        for dx in range(-sr, sr + 1):
            dist = 0.0
            for ty in range(-pr, pr + 1):
                for tx in range(-pr, pr + 1):
                    diff = px(i + ty, j + tx) - px(i + dy + ty, j + dx + tx)
                    dist += diff * diff
            w = np.exp(-dist / (patch * patch * h * h))
            num += w * px(i + dy, j + dx)
            den += w
    return num / den


def nlm_bruteforce(x: np.ndarray, patch: int = 5, search: int = 11,
                   h: float = 10.0) -> np.ndarray:
    """The literal definition evaluated pixel by pixel (tiny images only)."""
    out = np.empty(x.shape, dtype=np.float64)
    for i in range(x.shape[0]):
        for j in range(x.shape[1]):
            out[i, j] = nlm_pixel(x, i, j, patch, search, h)
    return out
