"""The seeded input generators: the separable Gaussian blur of the serving stream equals
the tap-by-tap 2-D circular convolution, and the generators are deterministic per seed."""
import numpy as np
import pytest

from paper_1805_02158_gb300 import synth


@pytest.mark.parametrize("k,s,shape", [(25, 1.6, (40, 36)), (7, 1.6, (27, 30)), (5, 1.2, (12, 18))])
def test_separable_gaussian_blur_equals_direct(k, s, shape):
    x = np.random.default_rng(k).uniform(0, 255, shape)
    t = synth.gaussian_taps(k, s)
    np.testing.assert_allclose(np.outer(t, t), synth.gaussian_psf(k, s), rtol=0, atol=1e-15)
    np.testing.assert_allclose(synth.circular_blur_separable(x, t, t),
                               synth.circular_blur_direct(x, synth.gaussian_psf(k, s)),
                               rtol=0, atol=1e-10)


def test_generators_are_deterministic_per_seed():
    a, b = synth.serving_request(3), synth.serving_request(3)
    assert a.task == b.task and a.height == b.height
    np.testing.assert_array_equal(a.y, b.y)
    c = synth.serving_request(4)
    assert c.y.shape != a.y.shape or not np.array_equal(c.y, a.y)
    u = synth.poisson_arrivals(200.0, 1000, seed=0)
    assert np.all(np.diff(u) > 0) and abs(u[-1] / 1000 - 1 / 200.0) < 0.2 / 200.0
