"""Pins for the oracle's vector extrapolation (Sec. III): MPE (Algorithm 1) with MGS
(Algorithm 2), RRE (Eq. (19)) and SVD-MPE.

The checks use mathematics the paper states, not the oracle's own code paths:
exactness on linear maps when kappa is the degree of the minimal polynomial (Eqs. (13)-
(16)), sum gamma = 1 (Eq. (11)), RRE as the constrained least-squares / KKT solution
(Eq. (19)), MPE as min ||U c|| with c_kappa = 1 (Eq. (18)) via a library least-squares
solver, SVD-MPE via a library SVD, Algorithm 1 step 4 against the direct weighted sum,
the MPE/RRE relation of Sec. III-B, the asymptotic rate of Eq. (20) and the breakdown
rule (MPE does not exist when sum c = 0)."""
import numpy as np
import pytest

from oracle import ve


def linear_sequence(A, b, x0, count):
    xs = [x0]
    for _ in range(count - 1):
        xs.append(A @ xs[-1] + b)
    return xs


def random_contraction(n, seed, radius=0.9):
    # well-separated real spectrum, so the Krylov columns of U stay resolvable
    rng = np.random.default_rng(seed)
    # (no eigenvalue near 0, whose mode would vanish after the m lead-in steps)
    mags = np.linspace(0.3, radius, n)
    lam = rng.permutation(mags * np.where(np.arange(n) % 2 == 0, 1.0, -1.0))
    V = rng.standard_normal((n, n)) + 3 * np.eye(n)
    return V @ np.diag(lam) @ np.linalg.inv(V), lam


@pytest.mark.parametrize("n", [6, 7, 8, 10])
@pytest.mark.parametrize("method", ["mpe", "rre", "svdmpe"])
@pytest.mark.parametrize("m", [0, 3])
def test_exact_fixed_point_when_kappa_is_dimension(n, method, m):
    A, _ = random_contraction(n, seed=n)
    rng = np.random.default_rng(100 + n)
    b = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    xstar = np.linalg.solve(np.eye(n) - A, b)
    xs = linear_sequence(A, b, x0, m + n + 2)[m:]
    x, gamma, info = ve.extrapolate(xs, method)
    assert not info["breakdown"]
    assert abs(gamma.sum() - 1.0) < 1e-13
    np.testing.assert_allclose(x, xstar, rtol=1e-8, atol=1e-8 * np.abs(xstar).max())


@pytest.mark.parametrize("method", ["mpe", "rre", "svdmpe"])
def test_exact_with_few_distinct_eigenvalues(method):
    # A diagonal in R^20 with 4 distinct eigenvalues: minimal polynomial degree 4.
    lam = np.repeat([0.9, -0.6, 0.3, 0.75], 5)
    A = np.diag(lam)
    rng = np.random.default_rng(7)
    b = rng.standard_normal(20)
    xs = linear_sequence(A, b, rng.standard_normal(20), 6)  # kappa = 4 -> 6 vectors
    x, gamma, info = ve.extrapolate(xs, method)
    np.testing.assert_allclose(x, b / (1 - lam), rtol=1e-9)
    # kappa = 3 is not enough
    x3, _, _ = ve.extrapolate(xs[:5], method)
    assert np.abs(x3 - b / (1 - lam)).max() > 1e-6


def test_gamma_sums_to_one_random():
    rng = np.random.default_rng(8)
    xs = [rng.standard_normal(50) for _ in range(7)]
    for method in ["mpe", "rre", "svdmpe"]:
        _, g, info = ve.extrapolate(xs, method)
        assert abs(g.sum() - 1.0) < 1e-14


def test_rre_is_kkt_solution():
    rng = np.random.default_rng(9)
    xs = [rng.standard_normal(40) for _ in range(6)]
    U = np.stack([xs[i + 1] - xs[i] for i in range(5)], 1)
    d = np.linalg.solve(U.T @ U, np.ones(5))
    _, g, _ = ve.extrapolate(xs, "rre")
    np.testing.assert_allclose(g, d / d.sum(), rtol=1e-10)
    # and it minimises ||U gamma|| over sum gamma = 1: random feasible perturbations do worse
    base = np.linalg.norm(U @ g)
    for _ in range(20):
        z = rng.standard_normal(5)
        z -= z.mean()
        assert np.linalg.norm(U @ (g + 1e-3 * z)) >= base


def test_mpe_is_constrained_least_squares():
    rng = np.random.default_rng(10)
    xs = [rng.standard_normal(40) for _ in range(6)]
    U = np.stack([xs[i + 1] - xs[i] for i in range(5)], 1)
    cp = np.linalg.lstsq(U[:, :4], -U[:, 4], rcond=None)[0]
    c = np.concatenate([cp, [1.0]])
    _, g, _ = ve.extrapolate(xs, "mpe")
    np.testing.assert_allclose(g, c / c.sum(), rtol=1e-10)


def test_svdmpe_uses_smallest_right_singular_vector():
    rng = np.random.default_rng(11)
    xs = [rng.standard_normal(40) for _ in range(6)]
    U = np.stack([xs[i + 1] - xs[i] for i in range(5)], 1)
    v = np.linalg.svd(U)[2][-1]
    _, g, _ = ve.extrapolate(xs, "svdmpe")
    np.testing.assert_allclose(g, v / v.sum(), rtol=1e-9)


def test_mgs_is_a_qr_factorisation():
    rng = np.random.default_rng(12)
    U = rng.standard_normal((30, 6))
    Q, R = ve.mgs_qr(U)
    np.testing.assert_allclose(Q @ R, U, atol=1e-12)
    np.testing.assert_allclose(Q.T @ Q, np.eye(6), atol=1e-12)
    assert np.allclose(np.tril(R, -1), 0) and np.all(np.diag(R) > 0)
    R_lib = np.linalg.qr(U)[1]
    np.testing.assert_allclose(np.abs(R), np.abs(R_lib), atol=1e-12)


@pytest.mark.parametrize("method", ["mpe", "rre", "svdmpe"])
def test_step4_equals_weighted_sum(method):
    rng = np.random.default_rng(13)
    xs = [rng.standard_normal(25) + 3 for _ in range(6)]
    x, g, _ = ve.extrapolate(xs, method)
    np.testing.assert_allclose(x, ve.combine_direct(xs, g), atol=1e-11)


def test_mpe_rre_relation():
    """mu_k x^RRE_k = mu_{k-1} x^RRE_{k-1} + nu_k x^MPE_k, mu_k = mu_{k-1} + nu_k, with
    mu = 1/||U gamma^RRE||^2 and nu = 1/||U gamma^MPE||^2 (all positive)."""
    rng = np.random.default_rng(14)
    for trial in range(4):
        xs = [rng.standard_normal(30) for _ in range(7)]
        for kap in (2, 3, 4, 5):
            sub = xs[:kap + 2]
            xr, gr, _ = ve.extrapolate(sub, "rre")
            xm, gm, _ = ve.extrapolate(sub, "mpe")
            xr1, gr1, _ = ve.extrapolate(sub[:-1], "rre")
            U = ve.difference_matrix(sub)
            mu = 1 / np.linalg.norm(U @ gr) ** 2
            mu1 = 1 / np.linalg.norm(U[:, :-1] @ gr1) ** 2
            nu = 1 / np.linalg.norm(U @ gm) ** 2
            assert mu > 0 and mu1 > 0 and nu > 0
            assert abs(mu - (mu1 + nu)) < 1e-10 * mu
            np.testing.assert_allclose(mu * xr, mu1 * xr1 + nu * xm, rtol=1e-9, atol=1e-9 * mu)


@pytest.mark.parametrize("method", ["mpe", "rre"])
def test_asymptotic_rate(method):
    """Eq. (20): x_(m,kappa) - x* = O(lambda_{kappa+1}^m) for diagonal A."""
    lam = np.array([0.95, 0.9, 0.85, 0.5, 0.45, 0.2, 0.1])
    A = np.diag(lam)
    b = np.ones(7)
    xstar = b / (1 - lam)
    kap = 3
    x0 = np.zeros(7)
    errs = {}
    for m in (10, 20, 30):
        xs = linear_sequence(A, b, x0, m + kap + 2)[m:]
        x, _, _ = ve.extrapolate(xs, method)
        errs[m] = np.linalg.norm(x - xstar)
    rate1 = (errs[20] / errs[10]) ** (1 / 10)
    rate2 = (errs[30] / errs[20]) ** (1 / 10)
    assert abs(rate2 - lam[kap]) < 0.03 and abs(rate1 - lam[kap]) < 0.06
    # FP itself converges at lambda_1 = 0.95: extrapolation is much faster
    assert errs[30] < 1e-3 * np.linalg.norm(linear_sequence(A, b, x0, 31)[30] - xstar)


def test_stability_sum_bounded():
    """Eq. (21): sum |gamma| stays bounded as m grows (linear, diagonalisable A)."""
    lam = np.array([0.9, 0.7, -0.5, 0.3, 0.1, 0.05])
    A = np.diag(lam)
    b = np.ones(6)
    sums = []
    for m in range(2, 22, 2):
        xs = linear_sequence(A, b, np.zeros(6), m + 2 + 2)[m:]
        _, g, info = ve.extrapolate(xs, "rre")
        sums.append(info["sum_abs_gamma"])
    # gamma tends to the normalised coefficients of (z - 0.9)(z - 0.7) = z^2 - 1.6 z + 0.63,
    # so sum |gamma| -> 3.23 / 0.03
    limit = (0.63 + 1.6 + 1.0) / abs(0.63 - 1.6 + 1.0)
    assert max(sums) < 2 * limit and abs(sums[-1] - limit) < 0.02 * limit


def test_breakdown_when_coefficients_sum_to_zero():
    # A pure drift x_i = x_0 + i v (A = I, no fixed point): u_0 = u_1, c = (-1, 1), sum 0.
    v = np.arange(1.0, 9.0)
    xs = [v * i for i in range(3)]
    x, g, info = ve.extrapolate(xs, "mpe")
    assert x is None and info["breakdown"]
    x, g, info = ve.extrapolate(xs, "rre")
    assert x is None and info["breakdown"]


def test_breakdown_on_zero_leading_difference():
    xs = [np.ones(5), np.ones(5), np.arange(5.0), np.arange(5.0) * 2]
    for method in ["mpe", "rre", "svdmpe"]:
        x, g, info = ve.extrapolate(xs, method)
        assert x is None and info["breakdown"] and 0 in info["rank_deficient"]


@pytest.mark.parametrize("scale", [1.0, 1e3, 1e-3])
def test_rank_loss_threshold_is_relative(scale):
    """Reading of the rank-loss rule: column i of U is dependent iff r_ii^2 <= 1e-12 |u_i|^2,
    a test on the relative remainder, unchanged by scaling U. A remainder of 1e-7 of the
    column (1e-14 squared) is dependent, one of 1e-5 (1e-10 squared) is not."""
    e1, e2, e3 = np.eye(3)
    for delta, dependent in [(1e-7, True), (1e-5, False)]:
        U = scale * np.stack([e1, e1 + delta * e2, e3], axis=1)
        Q, R = ve.mgs_qr(U)
        assert R[1, 1] == pytest.approx(scale * delta, rel=1e-6)
        assert (1 in ve.rank_deficient_columns(U, R)) is dependent
        assert 0 not in ve.rank_deficient_columns(U, R) and 2 not in ve.rank_deficient_columns(U, R)
