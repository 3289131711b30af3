"""Pins for the oracle's denoiser f(x) (non-local means; the role of f in Eq. (3)).

Checked against facts that do not come from the oracle's vectorised code: the literal
per-pixel definition, NumPy's own symmetric padding, and invariants of the definition
(constant images, shift equivariance, flips/transposition, convex-combination bounds,
and the h -> infinity / h -> 0 limits)."""
import numpy as np
import pytest

from oracle import nlm as N


def rand_img(seed, h, w):
    return np.random.default_rng(seed).uniform(0.0, 255.0, size=(h, w))


@pytest.mark.parametrize("shape", [(8, 8), (9, 7)])
def test_vectorised_matches_bruteforce(shape):
    x = rand_img(1, *shape)
    # smooth-ish image so that many weights are far from 0 and 1
    x = 0.5 * x + 0.5 * np.add.outer(np.arange(shape[0]) * 9.0, np.arange(shape[1]) * 7.0)
    f = N.nlm(x)
    g = N.nlm_bruteforce(x)
    np.testing.assert_allclose(f, g, rtol=1e-12, atol=1e-10)


def test_brute_force_small_patch_and_window():
    x = rand_img(2, 8, 8) * 0.1
    np.testing.assert_allclose(N.nlm(x, patch=3, search=5, h=3.0),
                               N.nlm_bruteforce(x, patch=3, search=5, h=3.0), rtol=1e-12)


def test_pixel_samples_on_larger_image():
    x = rand_img(3, 20, 24) * 0.3
    f = N.nlm(x)
    for (i, j) in [(0, 0), (19, 23), (10, 5), (3, 22)]:
        assert abs(f[i, j] - N.nlm_pixel(x, i, j)) < 1e-10


def test_mirror_padding_is_numpy_symmetric():
    x = rand_img(4, 8, 11)
    np.testing.assert_array_equal(N.pad_symmetric(x, 7), np.pad(x, 7, mode="symmetric"))
    assert list(N.mirror_index(np.array([-1, -2, 5, 6, 7]), 6)) == [0, 1, 5, 5, 4]


def test_constant_image_is_fixed():
    x = np.full((12, 10), 77.25)
    np.testing.assert_allclose(N.nlm(x), x, rtol=0, atol=1e-12)


def test_shift_equivariance():
    x = rand_img(5, 12, 12) * 0.2
    np.testing.assert_allclose(N.nlm(x + 37.0), N.nlm(x) + 37.0, rtol=0, atol=1e-9)


def test_flip_and_transpose_equivariance():
    x = rand_img(6, 10, 13) * 0.2
    f = N.nlm(x)
    np.testing.assert_allclose(N.nlm(x[::-1, :]), f[::-1, :], atol=1e-10)
    np.testing.assert_allclose(N.nlm(x[:, ::-1]), f[:, ::-1], atol=1e-10)
    np.testing.assert_allclose(N.nlm(x.T), f.T, atol=1e-10)


def test_output_is_convex_combination():
    x = rand_img(7, 16, 16)
    f = N.nlm(x)
    xp = N.pad_symmetric(x, 5)
    # each output lies within [min, max] of its 11x11 (mirrored) search window
    for i in range(16):
        for j in range(16):
            win = xp[i:i + 11, j:j + 11]
            assert win.min() - 1e-9 <= f[i, j] <= win.max() + 1e-9


def test_large_h_gives_window_mean():
    x = rand_img(8, 10, 9)
    xp = N.pad_symmetric(x, 5)
    mean = np.zeros_like(x)
    for dy in range(11):
        for dx in range(11):
            mean += xp[dy:dy + 10, dx:dx + 9]
    mean /= 121.0
    np.testing.assert_allclose(N.nlm(x, h=1e9), mean, rtol=0, atol=1e-6)


def test_small_h_gives_identity():
    x = rand_img(9, 10, 10)
    np.testing.assert_allclose(N.nlm(x, h=1e-3), x, rtol=0, atol=1e-9)


def test_weights_use_mean_squared_patch_distance():
    # Two-valued image where the weight of each candidate is known in closed form:
    # a vertical step edge; for the pixel far left of the edge, candidates whose patch
    # crosses the edge by c columns get distance c * 5 * delta^2 / 25.
    delta = 10.0
    x = np.zeros((11, 30))
    x[:, 15:] = delta
    i, j = 5, 9   # patches of candidates with dx in [-5, 5] cover columns up to 16
    f = N.nlm(x, h=10.0)[i, j]
    num = den = 0.0
    for dy in range(-5, 6):
        for dx in range(-5, 6):
            # columns of the candidate patch: j+dx-2 .. j+dx+2; count those >= 15
            c = sum(1 for t in range(-2, 3) if j + dx + t >= 15)
            w = np.exp(-(c * 5 * delta ** 2 / 25.0) / 100.0)
            num += w * (delta if j + dx >= 15 else 0.0)
            den += w
    assert abs(f - num / den) < 1e-12
