"""Pins for the oracle's FP step (Eq. (7)) and cycling driver (Algorithm 3) on small
synthetic problems.

The strongest check is exact: the FP recursion Eq. (6) says
grad l(x_{k+1}) + alpha (x_{k+1} - f(x_k)) = 0, so the gradient of the objective (Eq. (5))
at x_{k+1} equals alpha (f(x_k) - f(x_{k+1})). The gradient is formed from H and H^T
directly, so a dropped sigma^2, alpha or conjugate in the solve fails this test."""
import numpy as np
import pytest

from oracle import fp, red
from oracle import operators as ops
from oracle.nlm import nlm
from paper_1805_02158_gb300 import synth


def small_deblur(seed=0, side=24):
    return synth.make_deblur(seed, side, side, synth.uniform_psf(5), np.sqrt(2.0))


def small_sr(seed=0, side=24):
    return synth.make_sr(seed, side, side, synth.gaussian_psf(7, 1.6), 3, 5.0)


@pytest.mark.parametrize("make", [small_deblur, small_sr])
def test_fp_step_satisfies_first_order_recursion(make):
    p = make()
    F = fp.FPOperator(p.y, p.psf, p.y.shape if p.scale == 1 else (p.height, p.width), p.scale,
                      p.sigma, p.alpha, cg_iters=400)
    x = p.x0
    x1, fx = F.step_with_f(x)
    fx1 = nlm(x1)
    g = red.gradient(x1, fx1, p.y, F.otf, p.scale, p.sigma, p.alpha)
    expect = p.alpha * (fx - fx1)
    np.testing.assert_allclose(g, expect, rtol=1e-6, atol=1e-7 * np.abs(expect).max())


def test_fp_converges_and_gradient_vanishes():
    p = small_deblur(1)
    F = fp.FPOperator(p.y, p.psf, p.y.shape, 1, p.sigma, p.alpha)
    rcs = []
    x, st = red.solve(F, p.x0, "none", max_calls=120,
                      callback=lambda c, v: rcs.append(v.copy()))
    changes = [red.rel_change(rcs[i + 1], rcs[i]) for i in range(len(rcs) - 1)]
    # slow linear convergence (the reason for extrapolation), but steadily contracting
    assert changes[-1] < 0.03 * changes[0]
    assert changes[-1] < changes[len(changes) // 2]
    g = red.gradient(x, nlm(x), p.y, F.otf, 1, p.sigma, p.alpha)
    g0 = red.gradient(p.x0, nlm(p.x0), p.y, F.otf, 1, p.sigma, p.alpha)
    assert np.linalg.norm(g) < 1e-3 * np.linalg.norm(g0)


def test_driver_counts_and_termination():
    p = small_deblur(2, 16)
    F = fp.FPOperator(p.y, p.psf, p.y.shape, 1, p.sigma, p.alpha)
    calls = []
    x, st = red.solve(F, p.x0, "rre", m=0, kappa=4, max_calls=23, callback=lambda c, v: calls.append(c))
    assert st["fp_calls"] == 23 and calls == list(range(1, 24))
    assert st["ve_steps"] == 4  # after calls 5, 10, 15, 20
    x, st = red.solve(F, p.x0, "none", max_calls=500, tol=1e-3)
    assert st["fp_calls"] < 500 and st["rel_change"] < 1e-3
    # the FP iterate returned is F applied to the previous one
    x2, st2 = red.solve(F, p.x0, "none", max_calls=st["fp_calls"] - 1)
    np.testing.assert_allclose(F(x2), x, atol=1e-10)


def test_ve_reaches_fp_objective_in_fewer_calls():
    """Sec. IV: FP-MPE/RRE attains E(x*_FP) in fewer denoiser calls than FP."""
    p = small_deblur(3, 32)
    F = fp.FPOperator(p.y, p.psf, p.y.shape, 1, p.sigma, p.alpha)
    budget = 80
    xfp, _ = red.solve(F, p.x0, "none", max_calls=budget)
    e_fp = red.objective(xfp, nlm(xfp), p.y, F.otf, 1, p.sigma, p.alpha)
    for method in ("mpe", "rre"):
        reached = []

        def cb(c, v):
            if not reached and red.objective(v, nlm(v), p.y, F.otf, 1, p.sigma, p.alpha) <= e_fp:
                reached.append(c)
        red.solve(F, p.x0, method, m=0, kappa=4, max_calls=budget, callback=cb)
        assert reached and reached[0] < 0.75 * budget, (method, reached)


@pytest.mark.parametrize("make", [small_deblur, small_sr])
def test_objective_gradient_and_value_with_a_linear_denoiser(make):
    """Eq. (4) against Eq. (5) where the RED prior is a plain quadratic: with a symmetric
    linear denoiser f(x) = W x, rho(x) = x^T (x - W x) / 2 has gradient x - W x, so the
    objective's central differences must equal the gradient of Eq. (5); E(0) = |y|^2/(2 s^2).
    A dropped 1/2, sigma^2, alpha or transpose in either function fails this."""
    p = make()
    shape = (p.height, p.width)
    otf = ops.psf_otf(p.psf, shape)
    rng = np.random.default_rng(3)
    n = p.height * p.width
    A = rng.uniform(0, 1, (n, n))
    Wm = (A + A.T) / (2 * n)                       # symmetric, spectral radius < 1
    f = lambda v: (Wm @ v.ravel()).reshape(shape)  # noqa: E731
    x = rng.uniform(0, 255, shape)
    e = lambda v: red.objective(v, f(v), p.y, otf, p.scale, p.sigma, p.alpha)  # noqa: E731
    g = red.gradient(x, f(x), p.y, otf, p.scale, p.sigma, p.alpha)
    h = 1e-3
    for idx in [(0, 0), (3, 5), (p.height - 1, p.width - 2), (7, 11)]:
        d = np.zeros(shape)
        d[idx] = h
        num = (e(x + d) - e(x - d)) / (2 * h)
        assert abs(num - g[idx]) <= 1e-6 * max(1.0, abs(g[idx]))
    assert e(np.zeros(shape)) == pytest.approx(float(np.vdot(p.y, p.y)) / (2 * p.sigma ** 2),
                                               rel=1e-12)


def test_breakdown_continues_from_the_last_fp_iterate():
    """Reading: when an extrapolation does not exist the next cycle starts from the last FP
    iterate. A constant drift x -> x + c (all differences equal, so U has rank 1 and every
    extrapolation breaks down) must then advance by c at every call, as plain FP does."""
    c = np.linspace(0.5, 2.0, 6)

    class Drift:
        def __call__(self, x):
            return x + c

    x0 = np.ones(6)
    for method in ["mpe", "rre", "svdmpe"]:
        x, st = red.solve(Drift(), x0, method, m=1, kappa=3, max_calls=13)
        assert st["fp_calls"] == 13 and st["ve_steps"] == 2 and st["ve_breakdowns"] == 2
        np.testing.assert_allclose(x, x0 + 13 * c, rtol=1e-14)


def test_psnr_hand_computed():
    """PSNR = 10 log10(255^2 / MSE) with MSE the mean over all pixels (Sec. IV reports PSNR
    on the [0, 255] scale): values worked out by hand."""
    # MSE = 255^2 / 100 -> exactly 20 dB; MSE = 255^2 -> exactly 0 dB
    assert red.psnr(np.full((2, 2), 25.5), np.zeros((2, 2))) == pytest.approx(20.0, abs=1e-12)
    assert red.psnr(np.full(3, 255.0), np.zeros(3)) == pytest.approx(0.0, abs=1e-12)
    # errors (-2, 0, 3): MSE = 13 / 3, 255^2 / MSE = 195075 / 13 = 15005.769230769...,
    # log10 of it = 4 + log10(1.5) + log10(1.000384615...) = 4.1762582..., so 41.762583 dB
    assert red.psnr(np.array([10.0, 20.0, 30.0]), np.array([12.0, 20.0, 27.0])) == \
        pytest.approx(41.76258263, abs=1e-7)


def test_rel_change_hand_computed():
    """Termination test of Algorithm 3: ||x_new - x_old|| / ||x_old||. x_old = (0, 0, 10),
    x_new = (3, 4, 0): the difference has norm sqrt(125) = 11.18033988..., so the relative
    change is 1.118033988... (dividing by ||x_new|| = 5 would give 2.236...)."""
    assert red.rel_change(np.array([3.0, 4.0, 0.0]), np.array([0.0, 0.0, 10.0])) == \
        pytest.approx(1.1180339887498949, rel=1e-14)
    x = np.array([[1.0, -2.0], [2.0, 4.0]])
    assert red.rel_change(x, x) == 0.0


def test_ve_stop_tol_zero_and_huge_reduce_to_full_cycling_and_plain_fp():
    """ve_stop_tol = 0 never ends extrapolation (full cycling, bit for bit); a tolerance
    above every relative change ends it at the first FP step, after which the driver is the
    plain FP iteration of Eq. (7), bit for bit."""
    p = small_deblur(3, 20)
    F = fp.FPOperator(p.y, p.psf, p.y.shape, 1, p.sigma, p.alpha)
    x_full, st_full = red.solve(F, p.x0, "rre", kappa=4, max_calls=27)
    x0s, st0 = red.solve(F, p.x0, "rre", kappa=4, max_calls=27, ve_stop_tol=0.0)
    np.testing.assert_array_equal(x0s, x_full)
    assert st0["ve_stopped_at"] is None and st0["ve_steps"] == st_full["ve_steps"] == 5
    x_fp, _ = red.solve(F, p.x0, "none", max_calls=27)
    x_big, st_big = red.solve(F, p.x0, "mpe", kappa=4, max_calls=27, ve_stop_tol=1e30)
    np.testing.assert_array_equal(x_big, x_fp)
    assert st_big["ve_stopped_at"] == 1 and st_big["ve_steps"] == 0


def test_ve_stop_tol_hands_over_to_plain_fp_at_the_first_small_change():
    """Extrapolation ends at the first FP step whose relative change is below ve_stop_tol:
    the cycles completed before it extrapolated, and every later step is a plain FP step
    from that step's iterate (no extrapolation at the end of its cycle either)."""
    p = small_deblur(4, 20)
    F = fp.FPOperator(p.y, p.psf, p.y.shape, 1, p.sigma, p.alpha)
    seen = {}
    x, st = red.solve(F, p.x0, "rre", kappa=4, max_calls=60, ve_stop_tol=2e-3,
                      callback=lambda c, v: seen.__setitem__(c, v.copy()))
    s = st["ve_stopped_at"]
    assert s is not None and 5 < s < 60
    assert st["ve_steps"] == s // 5
    assert st["rel_change"] is not None
    x_tail, _ = red.solve(F, seen[s], "none", max_calls=60 - s)
    np.testing.assert_array_equal(x, x_tail)
    # before the stop every cycle's change stayed at or above the threshold
    _, st_hi = red.solve(F, p.x0, "rre", kappa=4, max_calls=s - 1, ve_stop_tol=2e-3)
    assert st_hi["ve_stopped_at"] is None
