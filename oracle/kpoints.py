"""Bloch-periodic Hamiltonian at a wavevector k (oracle, complex FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. evp of the periodic problem (Eq. ksproblemPer, Sec. 2.1): the
cell-periodic part u of a Bloch state at wavevector k solves

    (-1/2 lap - i k.grad + 1/2 |k|^2 + V) u = eps u,   u periodic on the box.

With real FE basis functions N_j the weak form gives, per cell,

    H_e(k) = 1/2 K_e - i (k . G_e) + 1/2 |k|^2 A_e + V_e,
    G_e^(d)_jl = int N_j d_d N_l,   A_e = int N_j N_l (consistent mass),

all by the cell's Gauss rule (the same quadrature as Eq. discreteHam).  The
assembled -i k.G is Hermitian because G^(d)_jl + G^(d)_lj integrates
d_d(N_j N_l), which vanishes over the periodic box; the assembled H(k) is then
brought to the standard form H~(k) = M^{-1/2} H(k) M^{-1/2} with the GLL mass
(Eq. hep).  On a uniform mesh K_e, G_e and A_e are the same for every cell, so
H_e(k) - H_e(0) = -i k.G + 1/2 |k|^2 A is one cell-independent matrix.

Scope: the local Hamiltonian; Bloch phases of the nonlocal projectors are
not modelled.
"""
from __future__ import annotations

import numpy as np


class BlochProblem:
    """H~(k) of a periodic oracle ``Problem`` without projectors."""

    def __init__(self, prob, k):
        if not prob.mesh.periodic:
            raise ValueError("Bloch states need a periodic box")
        if prob.C is not None:
            raise ValueError("projector Bloch phases are not modelled")
        self.prob = prob
        self.k = np.asarray(k, dtype=np.float64).reshape(3)
        b = prob.basis
        WN = b.W[:, None] * b.N
        self.G = [WN.T @ b.dN[:, :, d] for d in range(3)]      # int N_j d_d N_l
        self.A = WN.T @ b.N                                    # int N_j N_l
        kG = sum(self.k[d] * self.G[d] for d in range(3))
        self.shift = -1j * kG + 0.5 * float(self.k @ self.k) * self.A   # H_e(k) - H_e(0)

    @property
    def ndofs(self):
        """Number of unknowns M."""
        return self.prob.ndofs

    def cell_hamiltonian(self, e: int) -> np.ndarray:
        """H_e(k) = H_e(0) - i k.G + 1/2 |k|^2 A (Eq. evp in FE form)."""
        return self.prob.cell_hamiltonian(e) + self.shift

    def apply_Htilde(self, X: np.ndarray) -> np.ndarray:
        """H~(k) X for a complex block X (M x ncol)."""
        p = self.prob
        mesh = p.mesh
        Xs = p.minv_sqrt[:, None] * np.asarray(X, dtype=np.complex128)
        out = np.zeros_like(Xs)
        for e in range(mesh.ncells):
            d = mesh.cell_dofs(e)
            ok = d >= 0
            He = self.cell_hamiltonian(e)[np.ix_(ok, ok)]
            np.add.at(out, d[ok], He @ Xs[d[ok]])
        return p.minv_sqrt[:, None] * out

    def dense_Htilde(self) -> np.ndarray:
        """Dense H~(k) for tiny meshes (brute force)."""
        n = self.ndofs
        return self.apply_Htilde(np.eye(n, dtype=np.complex128))
