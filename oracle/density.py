"""Spectrum-splitting Rayleigh-Ritz and electron density (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 3.5 of arXiv:1903.10959, the steps right after the ChFSI step:

* Algorithm rr (spectrum splitting): with X the CholGS output, the projected
  Hamiltonian H^ = X^T H~ X, its N_fr largest eigenpairs H^ Q_fr = Q_fr D_fr,
  and the partial rotation X_fr = X Q_fr.
* Algorithm dc: the Fermi energy mu from the electron-count constraint
  2 (N_oc + sum_{i > N_oc} f(eps_i, mu)) = N_e, where N_oc = N - N_fr states
  are taken fully occupied and f is the Fermi-Dirac function
  1 / (1 + exp((eps - mu) / (k_B T))) (smearing of Sec. 3.2); then the density
  of Eq. elecDensSP,
      rho(x) = 2 n^T(x) [Psi_e Psi_e^T + Psi_fr,e (f(D_fr) - I) Psi_fr,e^T] n(x),
  with Psi = M^{-1/2} X and Psi_fr = M^{-1/2} X_fr restricted to a cell's
  nodes and n(x) the cell's basis functions.

Readings:
* The density is evaluated at the q^3 Gauss points of every cell, the points
  of the Hamiltonian integrals (the paper evaluates it at the quadrature points
  of its cells).  Output layout: rho[e, a + q (b + q c)], cells x fastest.
* Eigenvalues D_fr and the rotated columns come out ascending (the N_fr
  largest Ritz values in increasing order).
* The Fermi level is found by bisection on mu (the constraint is increasing
  in mu) to a relative width of 1e-15.
"""
from __future__ import annotations

import numpy as np


def rayleigh_ritz_split(apply_Ht, X: np.ndarray, n_fr: int):
    """Algorithm rr: (D_fr ascending, X_fr = X Q_fr) for the n_fr largest
    eigenpairs of H^ = X^T H~ X (X has orthonormal columns)."""
    X = np.asarray(X, dtype=np.float64)
    H = X.T @ apply_Ht(X)
    H = 0.5 * (H + H.T)
    w, Q = np.linalg.eigh(H)
    n = X.shape[1]
    sel = slice(n - n_fr, n)
    return w[sel], X @ Q[:, sel]


def fermi_dirac(eps, mu: float, kT: float):
    """f(eps, mu) = 1 / (1 + exp((eps - mu) / kT)) (Fermi-Dirac occupation)."""
    t = (np.asarray(eps, dtype=np.float64) - mu) / kT
    out = np.empty_like(t)
    pos = t > 0
    e = np.exp(-t[pos])
    out[pos] = e / (1.0 + e)
    out[~pos] = 1.0 / (1.0 + np.exp(t[~pos]))
    return out


def fermi_level(evals_fr, n_oc: int, n_electrons: float, kT: float):
    """Algorithm dc, step 1: mu with 2 (n_oc + sum f(eps_i, mu)) = N_e over the
    partially occupied Ritz values eps_i; returns (mu, f(eps_i, mu))."""
    eps = np.asarray(evals_fr, dtype=np.float64)

    def count(mu):
        """Electron count 2 (n_oc + sum f) at Fermi level mu."""
        return 2.0 * (n_oc + fermi_dirac(eps, mu, kT).sum())

    lo = eps.min() - 60.0 * kT
    hi = eps.max() + 60.0 * kT
    if not (count(lo) <= n_electrons <= count(hi)):
        raise ValueError("electron count outside what the states can hold")
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if count(mid) < n_electrons:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-15 * max(1.0, abs(mid)):
            break
    mu = 0.5 * (lo + hi)
    return mu, fermi_dirac(eps, mu, kT)


def density(prob, X: np.ndarray, X_fr: np.ndarray | None = None, occ_fr=None) -> np.ndarray:
    """Algorithm dc, steps 2-3 (Eq. elecDensSP) at the Gauss points of every cell:
    rho[e, q] = 2 sum_i psi_i(x_q)^2 + 2 sum_j (f_j - 1) psi_fr,j(x_q)^2."""
    s = prob.minv_sqrt[:, None]
    Psi = s * np.asarray(X, dtype=np.float64)
    Pfr = None
    if X_fr is not None and np.asarray(X_fr).shape[1] > 0:
        Pfr = s * np.asarray(X_fr, dtype=np.float64)
        w = 2.0 * (np.asarray(occ_fr, dtype=np.float64) - 1.0)
    N = prob.basis.N                                   # (q^3, n_e) basis values at the points
    dm = prob.mesh.dofmap()
    rho = np.zeros((prob.mesh.ncells, N.shape[0]))
    for e in range(prob.mesh.ncells):
        d = dm[e]
        ok = d >= 0
        vals = N[:, ok] @ Psi[d[ok]]                   # (q^3, n): psi_i at the points
        rho[e] = 2.0 * (vals ** 2).sum(axis=1)
        if Pfr is not None:
            vf = N[:, ok] @ Pfr[d[ok]]
            rho[e] += (vf ** 2) @ w
    return rho
