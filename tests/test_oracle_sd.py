"""Pins for the oracle's steepest-descent baseline of SD-MPE (Sec. IV-A, IV-B: a fixed-step
SD on the gradient of Eq. (5)) and for cycling with frozen gamma (Sec. III-C remark).

With a symmetric linear denoiser f(x) = W x the RED objective of Eq. (4) is exactly the
quadratic E(x) = |Hx - y|^2/(2 sigma^2) + alpha/2 x^T (I - W) x, whose Hessian and
minimiser are written out here as dense matrices built tap by tap (no FFT). On a linear
map with known eigenvalues the frozen-gamma cycles have a closed form."""
import numpy as np
import pytest

from oracle import red, sd
from oracle import operators as ops
from oracle.nlm import nlm
from paper_1805_02158_gb300 import synth
from test_oracle_linear import dense_blur_matrix, dense_decimation


def linear_denoiser(n, seed):
    """A symmetric W with non-negative entries (rows sum to about 1/2)."""
    A = np.random.default_rng(seed).uniform(0, 1, (n, n))
    return (A + A.T) / (2 * n)


def dense_problem(task, seed=0):
    """(y, psf, shape, scale, sigma, alpha, H) with H the dense degradation matrix."""
    rng = np.random.default_rng(seed)
    if task == "deblur":
        shape, psf, scale, sigma, alpha = (6, 6), synth.uniform_psf(3), 1, 1.0, 0.5
        H = dense_blur_matrix(psf, *shape)
    else:
        shape, psf, scale, sigma, alpha = (6, 6), synth.gaussian_psf(5, 1.2), 3, 1.0, 0.5
        H = dense_decimation(*shape, 3) @ dense_blur_matrix(psf, *shape)
    y = rng.uniform(0, 255, H.shape[0]).reshape(shape[0] // scale, shape[1] // scale)
    return y, psf, shape, scale, sigma, alpha, H


@pytest.mark.parametrize("task", ["deblur", "sr"])
def test_default_step_and_largest_hessian_eigenvalue(task):
    """mu = 1 / lambda_max(H^T H / sigma^2 + alpha I) for deblurring (exact), and a step no
    longer than that for super-resolution (H^T H = B^T S^T S B)."""
    for sigma, alpha in [(1.0, 0.5), (np.sqrt(2.0), 0.02), (5.0, 0.02)]:
        _, psf, shape, scale, _, _, H = dense_problem(task)
        n = shape[0] * shape[1]
        lam = np.linalg.eigvalsh(H.T @ H / sigma ** 2 + alpha * np.eye(n)).max()
        mu = sd.default_step(ops.psf_otf(psf, shape), sigma, alpha)
        if task == "deblur":
            assert 1.0 / mu == pytest.approx(lam, rel=1e-12)
        else:
            assert lam <= (1.0 / mu) * (1 + 1e-12)


@pytest.mark.parametrize("task", ["deblur", "sr"])
def test_sd_step_is_exact_descent_on_the_quadratic(task):
    """For the quadratic E, E(x - mu g) = E(x) - mu |g|^2 + mu^2/2 g^T A g with g = A x - b,
    A = H^T H/sigma^2 + alpha (I - W), b = H^T y/sigma^2: the SD step's value and its
    decrease are fixed by the dense A (a wrong sign, scale or transpose fails)."""
    y, psf, shape, scale, sigma, alpha, H = dense_problem(task, 1)
    n = shape[0] * shape[1]
    W = linear_denoiser(n, 2)
    A = H.T @ H / sigma ** 2 + alpha * (np.eye(n) - W)
    b = H.T @ y.ravel() / sigma ** 2
    f = lambda v: (W @ v.ravel()).reshape(shape)  # noqa: E731
    S = sd.SDOperator(y, psf, shape, scale, sigma, alpha, denoise=f)
    otf = S.otf
    E = lambda v: red.objective(v, f(v), y, otf, scale, sigma, alpha)  # noqa: E731
    x = np.random.default_rng(3).uniform(0, 255, shape)
    for _ in range(20):
        g = A @ x.ravel() - b
        x1 = S(x)
        np.testing.assert_allclose(x1.ravel(), x.ravel() - S.mu * g, rtol=1e-11, atol=1e-9)
        expect = E(x) - S.mu * g @ g + 0.5 * S.mu ** 2 * g @ A @ g
        assert E(x1) == pytest.approx(expect, rel=1e-10)
        assert E(x1) < E(x)
        x = x1


def spread_denoiser(n, seed):
    """A symmetric W = Q diag(w) Q^T with eigenvalues w spread over [0, 0.9]."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * rng.uniform(0.0, 0.9, n)) @ Q.T


@pytest.mark.parametrize("task,m,kappa", [("deblur", 0, 8), ("sr", 0, 4)])
def test_sd_and_sd_mpe_reach_the_dense_minimiser(task, m, kappa):
    """SD's fixed point is the minimiser A^{-1} b of the quadratic (12x12 images, alpha 0.05,
    which makes plain SD slow: its rate is 1 - mu lambda_min(A)); SD-MPE (Algorithm 3 with
    SD as the baseline) reaches the same point in several times fewer baseline steps.
    Deblurring uses the paper's m = 0, kappa = 8. For super-resolution the paper's
    m = 1, kappa = 10 exceeds what this 144-unknown problem resolves: its differences become
    dependent (r_ii^2 <= 1e-12 |u_i|^2) within 11 columns and every extrapolation is
    refused as rank-deficient, so kappa = 4 is used."""
    side, alpha, sigma = 12, 0.05, 1.0
    shape = (side, side)
    if task == "deblur":
        psf, scale = synth.gaussian_psf(5, 1.0), 1
        H = dense_blur_matrix(psf, side, side)
    else:
        psf, scale = synth.gaussian_psf(5, 1.2), 3
        H = dense_decimation(side, side, 3) @ dense_blur_matrix(psf, side, side)
    y = np.random.default_rng(4).uniform(0, 255, H.shape[0]).reshape(side // scale, side // scale)
    n = side * side
    W = spread_denoiser(n, 5)
    A = H.T @ H / sigma ** 2 + alpha * (np.eye(n) - W)
    x_star = np.linalg.solve(A, H.T @ y.ravel() / sigma ** 2).reshape(shape)
    f = lambda v: (W @ v.ravel()).reshape(shape)  # noqa: E731
    S = sd.SDOperator(y, psf, shape, scale, sigma, alpha, denoise=f)
    x0 = np.full(shape, 128.0)
    err = lambda v: np.linalg.norm(v - x_star) / np.linalg.norm(x_star)  # noqa: E731
    e_sd, e_mpe = [], []
    red.solve(S, x0, "none", max_calls=3000, callback=lambda c, v: e_sd.append(err(v)))
    assert e_sd[-1] < 1e-8
    red.solve(S, x0, "mpe", m=m, kappa=kappa, max_calls=600,
              callback=lambda c, v: e_mpe.append(err(v)))
    assert min(e_mpe) < 1e-10
    first = lambda e: next(i for i, v in enumerate(e) if v < 1e-6)  # noqa: E731
    assert first(e_mpe) < first(e_sd) / 5


def test_sd_mpe_accelerates_sd_with_nlm():
    """Sec. IV-A: SD-MPE needs fewer denoiser calls than SD to reach SD's objective after
    100 calls (24x24 deblurring, NLM denoiser, default step)."""
    p = synth.make_deblur(0, 24, 24, synth.uniform_psf(5), np.sqrt(2.0))
    S = sd.SDOperator(p.y, p.psf, p.y.shape, 1, p.sigma, p.alpha)
    E = lambda v: red.objective(v, nlm(v), p.y, S.otf, 1, p.sigma, p.alpha)  # noqa: E731
    x_sd, _ = red.solve(S, p.x0, "none", max_calls=100)
    target = E(x_sd)
    hist = []
    red.solve(S, p.x0, "mpe", m=0, kappa=8, max_calls=100, callback=lambda c, v: hist.append(v))
    reached = [c for c in range(10, 101, 10) if E(hist[c - 1]) <= target]
    assert reached and reached[0] < 100


def test_frozen_gamma_cycles_follow_the_closed_form():
    """On x -> diag(lam) x + b every extrapolation with weights gamma maps the error e of a
    cycle's start to lam^m P(lam) e, P(z) = sum_i gamma_i z^i (Eq. (11) with
    x_{m+i} - x* = lam^{m+i} e). With gamma frozen after the first cycle, c cycles and one
    more step give lam (lam^m P(lam))^c e_0; each frozen cycle takes m + kappa steps."""
    lam = np.array([-0.9, -0.6, -0.3, 0.1, 0.35, 0.5, 0.62, 0.7, 0.8, 0.88, 0.93, 0.97])
    b = np.linspace(-3.0, 5.0, lam.size)
    x_star = b / (1.0 - lam)

    class Linear:
        def __call__(self, x):
            return lam * x + b

    x0 = np.full(lam.size, 10.0)
    m, kappa, cycles = 2, 3, 4
    calls = (m + kappa + 1) + (cycles - 1) * (m + kappa) + 1
    x, st = red.solve(Linear(), x0, "mpe", m=m, kappa=kappa, max_calls=calls, freeze_after=1)
    assert st["fp_calls"] == calls and st["ve_steps"] == cycles
    assert st["frozen_steps"] == cycles - 1 and len(st["gammas"]) == 1
    gamma = st["gammas"][0]
    P = sum(g * lam ** i for i, g in enumerate(gamma))
    expect = x_star + lam * (lam ** m * P) ** cycles * (x0 - x_star)
    np.testing.assert_allclose(x, expect, rtol=1e-12, atol=1e-12)
    # full cycling recomputes gamma every cycle, which leaves the closed form
    x_full, st_full = red.solve(Linear(), x0, "mpe", m=m, kappa=kappa,
                                max_calls=(m + kappa + 1) * cycles + 1)
    assert st_full["frozen_steps"] == 0 and len(st_full["gammas"]) == cycles
    assert np.abs(x_full - expect).max() > 1e-6 * np.abs(expect).max()
