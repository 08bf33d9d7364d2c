"""Chebyshev-filtered subspace iteration (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The three sub-steps of step 7 of Algorithm scf in arXiv:1903.10959:
  7a CF      -- Chebyshev filter T_m(H-bar) X (Eq. chebFilter, Sec. 3.3) with
                H-bar = (H~ - c) / e mapping the unwanted interval [a, b]
                to [-1, 1];
  7b CholGS  -- S = X^T X, S = L L^T, L^{-1}, X <- X L^{-T}
                (Algorithm CholGS, Sec. 3.4);
  7c RR      -- H^ = X^T H~ X, H^ Q = Q D (ascending), X <- X Q (Sec. 3.5).

Readings of points the paper leaves open:
* The recurrence is the scaled (sigma-normalised) form of Zhou & Saad
  (the paper's reference for the filter): the result is
  T_m(H-bar) X / T_m((a0 - c) / e), which differs from Eq. chebFilter by one
  global scalar and keeps all values O(1).
* Bounds: b from a k-step Lanczos run (b = largest Ritz value of the
  tridiagonal + |beta_k|); a = largest and a0 = smallest Ritz value of the
  previous Rayleigh-Ritz step.
* Gamma point only: the Hermitian transposes of the paper become transposes.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def chebyshev_filter(apply_Ht, X: np.ndarray, m: int, a: float, b: float, a0: float):
    """Scaled degree-m Chebyshev filter (Eq. chebFilter; scaled form of Zhou & Saad).

    Y_1 = (s_1 / e)(H~ - c) X, Y_{k+1} = (2 s_{k+1} / e)(H~ - c) Y_k - s_k s_{k+1} Y_{k-1},
    s_1 = e / (a0 - c), s_{k+1} = 1 / (2 / s_1 - s_k), c = (a + b) / 2, e = (b - a) / 2.
    """
    if m < 1:
        return X.copy()
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    s1 = e / (a0 - c)
    s = s1
    Yprev = X
    Y = (s1 / e) * (apply_Ht(X) - c * X)
    for _ in range(2, m + 1):
        snew = 1.0 / (2.0 / s1 - s)
        Ynew = (2.0 * snew / e) * (apply_Ht(Y) - c * Y) - (s * snew) * Yprev
        Yprev, Y, s = Y, Ynew, snew
    return Y


def filter_scalars(m: int, a: float, b: float, a0: float):
    """(alpha_k, beta_k) of each recurrence step: Y_k = alpha_k (H~ - c) Y_{k-1} + beta_k Y_{k-2}."""
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    s1 = e / (a0 - c)
    out = [(s1 / e, 0.0)]
    s = s1
    for _ in range(2, m + 1):
        snew = 1.0 / (2.0 / s1 - s)
        out.append((2.0 * snew / e, -s * snew))
        s = snew
    return c, out


def exact_filter(evals: np.ndarray, evecs: np.ndarray, X: np.ndarray, m: int, a, b, a0):
    """Q p(Lambda) Q^T X with p(t) = T_m((t - c)/e) / T_m((a0 - c)/e), T_m evaluated
    by numpy's Chebyshev series (independent of the three-term recurrence)."""
    from numpy.polynomial import chebyshev as C
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    coef = np.zeros(m + 1)
    coef[m] = 1.0
    pv = C.chebval((evals - c) / e, coef) / C.chebval((a0 - c) / e, coef)
    return evecs @ (pv[:, None] * (evecs.T @ X))


def cholgs(X: np.ndarray):
    """Algorithm CholGS: S = X^T X; S = L L^T; L^{-1}; X^o = X L^{-T}."""
    S = X.T @ X
    L = np.linalg.cholesky(S)
    Linv = sla.solve_triangular(L, np.eye(len(S)), lower=True)
    return X @ Linv.T


def rayleigh_ritz(apply_Ht, X: np.ndarray):
    """Sec. 3.5: H^ = X^T H~ X; H^ Q = Q D, D ascending; X^R = X Q.  Returns (D, X^R)."""
    Hh = X.T @ apply_Ht(X)
    Hh = 0.5 * (Hh + Hh.T)
    D, Q = np.linalg.eigh(Hh)
    return D, X @ Q


def lanczos_upper_bound(apply_Ht, v0: np.ndarray, k: int) -> float:
    """k-step Lanczos on H~ from v0: b = max eig(T_k) + |beta_k| (bound of Zhou & Saad).

    Parity unpinned beyond b >= lambda_max: the bound is a heuristic.
    """
    v = v0 / np.linalg.norm(v0)
    vprev = np.zeros_like(v)
    alpha, beta = [], []
    bprev = 0.0
    for _ in range(k):
        w = apply_Ht(v) - bprev * vprev
        al = float(w @ v)
        w = w - al * v
        bt = float(np.linalg.norm(w))
        alpha.append(al)
        beta.append(bt)
        if bt == 0.0:
            break
        vprev, v, bprev = v, w / bt, bt
    T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    return float(np.linalg.eigvalsh(T)[-1] + abs(beta[-1]))


def residual_norms(apply_Ht, X: np.ndarray, evals: np.ndarray) -> np.ndarray:
    """r_i = ||H~ x_i - lambda_i x_i||_2 / ||x_i||_2 (standard form of Eq. hep)."""
    R = apply_Ht(X) - X * evals[None, :]
    return np.linalg.norm(R, axis=0) / np.linalg.norm(X, axis=0)


def generalized_residual_norms(apply_Ht, X: np.ndarray, evals, mass: np.ndarray):
    """||H Psi_i - lambda_i M Psi_i||_2 with Psi_i = M^{-1/2} x_i, x_i of unit norm
    (so Psi_i is M-normalised): equals ||M^{1/2} (H~ x_i - lambda_i x_i)||."""
    Xn = X / np.linalg.norm(X, axis=0)[None, :]
    R = apply_Ht(Xn) - Xn * evals[None, :]
    return np.linalg.norm(np.sqrt(mass)[:, None] * R, axis=0)


def chfsi(apply_Ht, X0: np.ndarray, m: int, iters: int, b: float, history=False):
    """ChFSI loop (step 7 of Algorithm scf, repeated): iteration 0 orthonormalises the
    start block and runs RR to get (a, a0); each later iteration filters with the
    previous bounds, then CholGS, then RR.  Returns (D, X[, per-iteration D])."""
    X = cholgs(np.array(X0, dtype=np.float64))
    D, X = rayleigh_ritz(apply_Ht, X)
    hist = [D.copy()]
    for _ in range(iters):
        a, a0 = float(D[-1]), float(D[0])
        X = chebyshev_filter(apply_Ht, X, m, a, b, a0)
        X = cholgs(X)
        D, X = rayleigh_ritz(apply_Ht, X)
        hist.append(D.copy())
    return (D, X, hist) if history else (D, X)
