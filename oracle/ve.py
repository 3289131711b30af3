"""Vector extrapolation in FP64 (Sec. III-B): MPE (Algorithm 1) with the modified
Gram-Schmidt QR of Algorithm 2, RRE (Eq. (19)) and SVD-MPE.

Notation follows the paper: from kappa + 2 iterates x_m, ..., x_{m+kappa+1} form
U = [u_0, ..., u_kappa], u_i = x_{m+i+1} - x_{m+i} (N x (kappa+1)); U = Q R.
The extrapolated vector is x_(m,kappa) = sum_{i=0}^{kappa} gamma_i x_{m+i} with
sum gamma_i = 1 (Eq. (11)), evaluated as in steps 3-4 of Algorithm 1:
xi_0 = 1 - gamma_0, xi_j = xi_{j-1} - gamma_j; eta = R_{kappa-1} xi;
x_(m,kappa) = x_m + Q_{kappa-1} eta.

Readings where the paper is silent (the same rules are used by the CUDA path):
  * Rank loss: column i of U is treated as dependent on the previous ones when
    r_ii^2 <= RANK_TOL * ||u_i||^2 (or u_i = 0).
      - in one of the first kappa columns: no extrapolation exists (breakdown);
      - only in the last column: MPE is unaffected (step 2 of Algorithm 1 does not use
        r_{kappa+1,kappa+1}); RRE's minimiser is then the MPE solution, which makes
        U gamma = 0.
  * MPE / SVD-MPE do not exist when the coefficients sum to zero (Sec. III-B remark);
    treated as |sum c| <= SUM_TOL * sum |c|.
  * On breakdown the caller continues from the last FP iterate.
Algorithm 1 step 2 writes sum_{i=0}^{k} c_i; the sum runs over i = 0..kappa with
c_kappa = 1.
"""
from __future__ import annotations

import numpy as np

RANK_TOL = 1e-12
SUM_TOL = 1e-12


def difference_matrix(xs) -> np.ndarray:
    """U of Algorithm 1 step 1 from the kappa+2 iterates (each flattened)."""
    X = np.stack([np.asarray(x, dtype=np.float64).ravel() for x in xs], axis=1)
    return X[:, 1:] - X[:, :-1]


def mgs_qr(U: np.ndarray):
    """Algorithm 2: modified Gram-Schmidt, U = Q R with R upper triangular and
    r_ii = ||u_i^{(i)}||_2 >= 0. A column whose remainder is exactly zero gets q_i = 0."""
    n, k = U.shape
    Q = np.zeros((n, k))
    R = np.zeros((k, k))
    for i in range(k):
        v = U[:, i].copy()
        for j in range(i):
            R[j, i] = float(Q[:, j] @ v)
            v = v - R[j, i] * Q[:, j]
        R[i, i] = float(np.linalg.norm(v))
        if R[i, i] > 0.0:
            Q[:, i] = v / R[i, i]
    return Q, R


def rank_deficient_columns(U: np.ndarray, R: np.ndarray):
    norms2 = np.einsum("ij,ij->j", U, U)
    return [i for i in range(R.shape[0])
            if norms2[i] == 0.0 or R[i, i] ** 2 <= RANK_TOL * norms2[i]]


def back_substitute(Rt: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve an upper-triangular system by back substitution."""
    k = Rt.shape[0]
    x = np.zeros(k)
    for i in range(k - 1, -1, -1):
        x[i] = (b[i] - Rt[i, i + 1:] @ x[i + 1:]) / Rt[i, i]
    return x


def forward_substitute(Lt: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve a lower-triangular system by forward substitution."""
    k = Lt.shape[0]
    x = np.zeros(k)
    for i in range(k):
        x[i] = (b[i] - Lt[i, :i] @ x[:i]) / Lt[i, i]
    return x


def mpe_coefficients(R: np.ndarray):
    """Algorithm 1 step 2: R_{kappa-1} c' = -r_{kappa+1}, c_kappa = 1. Returns c."""
    kap = R.shape[0] - 1
    if kap == 0:
        return np.array([1.0])
    cp = back_substitute(R[:kap, :kap], -R[:kap, kap])
    return np.concatenate([cp, [1.0]])


def mpe_gamma(R: np.ndarray):
    c = mpe_coefficients(R)
    s = c.sum()
    if abs(s) <= SUM_TOL * np.abs(c).sum():
        return None
    return c / s


def rre_gamma(R: np.ndarray):
    """RRE: R^T R d = 1 by forward then backward substitution, gamma = d / sum d."""
    ones = np.ones(R.shape[0])
    z = forward_substitute(R.T, ones)
    d = back_substitute(R, z)
    return d / d.sum()


def svdmpe_gamma(R: np.ndarray):
    """SVD-MPE: gamma = v_{kappa+1} / sum_i v_{i,kappa+1}, v_{kappa+1} the right singular
    vector of R for its smallest singular value."""
    _, _, vt = np.linalg.svd(R)
    v = vt[-1, :]
    s = v.sum()
    if abs(s) <= SUM_TOL * np.abs(v).sum():
        return None
    return v / s


def combine_qr(x_m: np.ndarray, Q: np.ndarray, R: np.ndarray, gamma: np.ndarray) -> np.ndarray:
    """Algorithm 1 steps 3-4: x_(m,kappa) = x_m + Q_{kappa-1} R_{kappa-1} xi."""
    kap = R.shape[0] - 1
    xi = 1.0 - np.cumsum(gamma[:kap])
    eta = R[:kap, :kap] @ xi
    return x_m + Q[:, :kap] @ eta


def extrapolate(xs, method: str = "mpe"):
    """One extrapolation from kappa + 2 iterates. Returns (x_new, gamma, info); on
    breakdown x_new and gamma are None and info['breakdown'] is True."""
    xs = [np.asarray(x, dtype=np.float64) for x in xs]
    shape = xs[0].shape
    U = difference_matrix(xs)
    Q, R = mgs_qr(U)
    kap = R.shape[0] - 1
    bad = rank_deficient_columns(U, R)
    info = {"R": R, "kappa": kap, "rank_deficient": bad, "breakdown": False}
    if any(i < kap for i in bad):
        info["breakdown"] = True
        return None, None, info
    if method == "mpe":
        gamma = mpe_gamma(R)
    elif method == "rre":
        gamma = mpe_gamma(R) if kap in bad else rre_gamma(R)
    elif method == "svdmpe":
        gamma = svdmpe_gamma(R)
    else:
        raise ValueError(method)
    if gamma is None:
        info["breakdown"] = True
        return None, None, info
    x_new = combine_qr(xs[0].ravel(), Q, R, gamma).reshape(shape)
    info["sum_abs_gamma"] = float(np.abs(gamma).sum())
    return x_new, gamma, info


def combine_direct(xs, gamma) -> np.ndarray:
    """Eq. (11): sum_{i=0}^{kappa} gamma_i x_{m+i}."""
    out = np.zeros_like(np.asarray(xs[0], dtype=np.float64))
    for g, x in zip(gamma, xs[: len(gamma)]):
        out = out + g * np.asarray(x, dtype=np.float64)
    return out
