"""Discrete Hamiltonian of a fixed effective potential (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Local part: H_e = 1/2 K_e + V_e per cell (Eq. discreteHam).
* Nonlocal part: H^nl_jk = sum_k C_{k,j} h_k C_{k,k'} with
  C_{k,j} = int chi_k N_j (Eqs. nlps, nonlocalHamDiscrete).
* Standard form: H~ = M^{-1/2} H M^{-1/2} (Eq. hep).

The effective potential is a sum of attractive Gaussian wells
V(x) = -sum_a D_a exp(-|x - R_a|^2 / (2 w_a^2)); every well is summed over
its image shifts {-1, 0, 1} L along each periodic axis (27 images when all
three are periodic).
Projectors are chi(r) = g(r) {1, x/s, y/s, z/s}, g = exp(-r^2 / (2 s^2)) for
r <= r_c and 0 beyond (one s-like and three p-like channels per site, the
l, m structure of Eq. nlps), r measured to the nearest periodic image.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .fe import CellBasis, Mesh, assemble_mass_diag, periodic_axes


def gaussian_wells(x: np.ndarray, centres, depths, widths, L: float, periodic):
    """V at points x (n, 3): -sum_a D_a exp(-|x - R_a - shift|^2 / (2 w_a^2)),
    shifts over the images along the periodic axes."""
    x = np.asarray(x, dtype=np.float64)
    v = np.zeros(len(x))
    per = periodic_axes(periodic)
    shifts = itertools.product(*[(-1, 0, 1) if pa else (0,) for pa in per])
    shifts = [np.array(s, dtype=np.float64) * L for s in shifts]
    for R, D, w in zip(np.asarray(centres), np.asarray(depths), np.asarray(widths)):
        for s in shifts:
            d = x - (R + s)
            v -= D * np.exp(-np.sum(d * d, axis=1) / (2.0 * w * w))
    return v


def harmonic(x: np.ndarray, centre, omega: float):
    """V = 1/2 omega^2 |x - c|^2 (used by the oscillator pin)."""
    d = np.asarray(x) - np.asarray(centre)
    return 0.5 * omega * omega * np.sum(d * d, axis=1)


class Problem:
    """Mesh + basis + potential: the data of Eq. kohnShamSolve for fixed V_eff."""

    def __init__(self, ncell, p, L, periodic, potential, projectors=None, q=None):
        """``potential``: callable V(points (n,3)) -> (n,).  ``projectors``:
        optional dict(centres (ns,3), sigma, rcut, h (ns,4))."""
        self.mesh = Mesh(ncell, p, L, periodic)
        self.basis = CellBasis(p, self.mesh.h, q)
        self.potential = potential
        self.K = self.basis.stiffness()
        self.mass = assemble_mass_diag(self.mesh, self.basis)
        self.minv_sqrt = 1.0 / np.sqrt(self.mass)
        self._cellH = {}
        self.C = None
        self.hnl = None
        if projectors is not None and len(projectors["centres"]):
            self.C, self.hnl = projector_matrix(self, **projectors)

    @property
    def ndofs(self):
        """Number of unknowns M (size of Eq. hep)."""
        return self.mesh.ndofs

    def cell_hamiltonian(self, e: int) -> np.ndarray:
        """H_e = 1/2 K_e + V_e for cell e (Eq. discreteHam)."""
        if e not in self._cellH:
            xq = self.basis.quad_coords(self.mesh.cell_origin(e))
            self._cellH[e] = 0.5 * self.K + self.basis.potential_matrix(self.potential(xq))
        return self._cellH[e]

    def apply_H(self, X: np.ndarray) -> np.ndarray:
        """H X = sum_e P_e^T H_e P_e X  (+ C h C^T X)  (Eqs. discreteHam, nonlocalHamDiscrete)."""
        X = np.asarray(X, dtype=np.float64)
        out = np.zeros_like(X)
        for e in range(self.mesh.ncells):
            d = self.mesh.cell_dofs(e)
            ok = d >= 0
            He = self.cell_hamiltonian(e)[np.ix_(ok, ok)]
            out[d[ok]] += He @ X[d[ok]]
        if self.C is not None:
            out += self.C.T @ (self.hnl[:, None] * (self.C @ X)) if X.ndim == 2 else \
                self.C.T @ (self.hnl * (self.C @ X))
        return out

    def apply_Htilde(self, X: np.ndarray) -> np.ndarray:
        """H~ X = M^{-1/2} H M^{-1/2} X (Eq. hep)."""
        s = self.minv_sqrt if X.ndim == 1 else self.minv_sqrt[:, None]
        return s * self.apply_H(s * X)

    def apply_Htilde_cells(self, cells, X: np.ndarray) -> np.ndarray:
        """Local part of H~ X over a subset of cells (the cell loop one task of a
        domain decomposition runs on its own cells, Sec. 3.7):
        M^{-1/2} sum_{e in cells} P_e^T H_e P_e M^{-1/2} X.  Summed over a
        partition of the cells it gives the local part of apply_Htilde."""
        s = self.minv_sqrt[:, None]
        Xs = s * np.asarray(X, dtype=np.float64)
        out = np.zeros_like(Xs)
        for e in cells:
            d = self.mesh.cell_dofs(int(e))
            ok = d >= 0
            He = self.cell_hamiltonian(int(e))[np.ix_(ok, ok)]
            out[d[ok]] += He @ Xs[d[ok]]
        return s * out

    def apply_Htilde_rows(self, rows, X: np.ndarray) -> np.ndarray:
        """Rows ``rows`` of H~ X, summing only the cells that contain them (for
        sampled checks on meshes too large for a full oracle apply)."""
        if not hasattr(self, "_node_cells"):
            dm = self.mesh.dofmap()
            inv = {}
            for e in range(self.mesh.ncells):
                for l, g in enumerate(dm[e]):
                    if g >= 0:
                        inv.setdefault(int(g), []).append((e, l))
            self._node_cells, self._dm = inv, dm
        s = self.minv_sqrt
        out = np.zeros((len(rows), X.shape[1]))
        for ii, j in enumerate(rows):
            for e, l in self._node_cells[int(j)]:
                d = self._dm[e]
                ok = d >= 0
                out[ii] += self.cell_hamiltonian(e)[l, ok] @ (s[d[ok], None] * X[d[ok]])
        if self.C is not None:
            Z = self.C @ (s[:, None] * X)
            out += self.C[:, np.asarray(rows)].T @ (self.hnl[:, None] * Z)
        return s[np.asarray(rows), None] * out

    def dense_H(self) -> np.ndarray:
        """Assembled H (small meshes only)."""
        n = self.ndofs
        H = np.zeros((n, n))
        for e in range(self.mesh.ncells):
            d = self.mesh.cell_dofs(e)
            ok = d >= 0
            H[np.ix_(d[ok], d[ok])] += self.cell_hamiltonian(e)[np.ix_(ok, ok)]
        if self.C is not None:
            Cd = self.C.toarray()
            H += Cd.T @ (self.hnl[:, None] * Cd)
        return H

    def dense_Htilde(self) -> np.ndarray:
        """Assembled H~ = M^{-1/2} H M^{-1/2} (Eq. hep; small meshes only)."""
        s = self.minv_sqrt
        return s[:, None] * self.dense_H() * s[None, :]

    def sparse_Htilde(self):
        """H~ as a scipy sparse matrix (medium meshes, e.g. the oscillator pin)."""
        rows, cols, vals = [], [], []
        for e in range(self.mesh.ncells):
            d = self.mesh.cell_dofs(e)
            ok = d >= 0
            He = self.cell_hamiltonian(e)[np.ix_(ok, ok)]
            dd = d[ok]
            rows.append(np.repeat(dd, len(dd)))
            cols.append(np.tile(dd, len(dd)))
            vals.append(He.ravel())
        H = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.ndofs, self.ndofs))
        if self.C is not None:
            H = H + self.C.T @ sp.diags(self.hnl) @ self.C
        S = sp.diags(self.minv_sqrt)
        return (S @ H @ S).tocsr()


def _min_image(d: np.ndarray, L: float, periodic) -> np.ndarray:
    per = np.array(periodic_axes(periodic))
    return np.where(per[None, :], d - L * np.round(d / L), d)


def projector_values(x: np.ndarray, centre, sigma: float, rcut: float, L: float,
                     periodic) -> np.ndarray:
    """chi_{s,k}(x) for the 4 channels at points x: (n, 4) (Eq. nlps form)."""
    d = _min_image(np.asarray(x) - np.asarray(centre), L, periodic)
    r2 = np.sum(d * d, axis=1)
    g = np.exp(-r2 / (2.0 * sigma * sigma)) * (r2 <= rcut * rcut)
    return np.stack([g, g * d[:, 0] / sigma, g * d[:, 1] / sigma, g * d[:, 2] / sigma], axis=1)


def projector_matrix(prob: Problem, centres, sigma, rcut, h):
    """C_{k,j} = int chi_k N_j by the Gauss rule of the cell (Eq. nonlocalHamDiscrete),
    assembled over every cell; returns (C as CSR (nproj x M), h flattened)."""
    mesh, basis = prob.mesh, prob.basis
    centres = np.asarray(centres, dtype=np.float64)
    ns = len(centres)
    rows, cols, vals = [], [], []
    for e in range(mesh.ncells):
        xq = basis.quad_coords(mesh.cell_origin(e))
        d = mesh.cell_dofs(e)
        ok = d >= 0
        for s in range(ns):
            chi = projector_values(xq, centres[s], sigma, rcut, mesh.L, mesh.per)
            if not np.any(chi):
                continue
            ce = (basis.W[:, None, None] * basis.N[:, :, None] * chi[:, None, :]).sum(0)  # (ne, 4)
            for k in range(4):
                rows.append(np.full(ok.sum(), 4 * s + k))
                cols.append(d[ok])
                vals.append(ce[ok, k])
    if rows:
        C = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(4 * ns, mesh.ndofs))
    else:
        C = sp.csr_matrix((4 * ns, mesh.ndofs))
    C.sum_duplicates()
    return C, np.asarray(h, dtype=np.float64).reshape(-1)


def wells_problem(ncell, p, L, periodic, centres, depths, widths, projectors=None, q=None):
    """Problem with V_eff = sum of Gaussian wells (the synthetic workloads)."""
    c = np.asarray(centres, dtype=np.float64)
    dpt = np.asarray(depths, dtype=np.float64)
    wd = np.asarray(widths, dtype=np.float64)
    return Problem(ncell, p, L, periodic,
                   lambda x: gaussian_wells(x, c, dpt, wd, L, periodic), projectors, q)
