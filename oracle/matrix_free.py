"""Matrix-free (sum-factorised) cell apply and its flop count (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper applies H through stored cell matrices and notes (Sec. 3.3.1,
footnote on the cell-level products) that a matrix-free evaluation is the
alternative.  On the tensor-product cell, with the 1-D GLL Lagrange basis
l_i, the Gauss rule (x_a, w_a) of the cell integrals and jac = h / 2, the
action of H_e = 1/2 K_e + V_e (Eq. discreteHam) factors into 1-D contractions
along the three axes:

    K_e u = (S (x) A (x) A + A (x) S (x) A + A (x) A (x) S) u,
        A_il = jac sum_a w_a l_i(x_a) l_l(x_a)      (1-D consistent mass),
        S_il = (1 / jac) sum_a w_a l_i'(x_a) l_l'(x_a)   (1-D stiffness),
    V_e u = (B^T (x) B^T (x) B^T) diag(W V) (B (x) B (x) B) u,
        B_al = l_l(x_a),  W = w_a w_b w_c jac^3.

Cell vectors are laid out [k][j][i] (local node i + n1 (j + n1 k), x fastest).
A contraction of one axis of length n_in into n_out with D values on the other
axes costs 2 n_out n_in D flops; ``flops_per_cell`` adds them up for the order
used here (the kinetic part shares the z and y passes between its three
terms), to compare with the dense cell product's 2 n_e^2 flops per vector.
"""
from __future__ import annotations

import numpy as np

from .fe import gauss_rule, gll_rule, lagrange_derivs, lagrange_values

_EIN = {0: "ai,kjic->kjac", 1: "aj,kjic->kaic", 2: "ak,kjic->ajic"}   # axis 0 = x, 1 = y, 2 = z


class Counter:
    """Running flop count of the contractions of one apply."""

    def __init__(self):
        self.flops = 0


def _contract(T: np.ndarray, X: np.ndarray, axis: int, cnt: Counter | None) -> np.ndarray:
    """Apply T (n_out x n_in) along one spatial axis of X (shape (z, y, x, ncol))."""
    if cnt is not None:
        other = X.size // X.shape[2 - axis]
        cnt.flops += 2 * T.shape[0] * T.shape[1] * other
    return np.einsum(_EIN[axis], T, X)


class MatrixFreeCell:
    """The 1-D factors of one cell (side h, degree p, q Gauss points per direction)."""

    def __init__(self, p: int, h: float, q: int | None = None):
        self.p, self.n1 = p, p + 1
        self.q = q if q is not None else p + 2
        nodes, _ = gll_rule(p)
        xq, wq = gauss_rule(self.q)
        jac = h / 2.0
        self.B = lagrange_values(nodes, xq)                  # (q, n1)
        dB = lagrange_derivs(nodes, xq)
        self.A = jac * (self.B * wq[:, None]).T @ self.B     # (n1, n1)
        self.S = (dB * wq[:, None]).T @ dB / jac
        w3 = wq[:, None, None] * wq[None, :, None] * wq[None, None, :]   # [c][b][a]
        self.W = w3 * jac ** 3

    def apply(self, u: np.ndarray, vq: np.ndarray, cnt: Counter | None = None) -> np.ndarray:
        """H_e u for cell vectors u (n_e x ncol, local order) and V at the q^3 Gauss
        points (point a + q (b + q c))."""
        n1, q = self.n1, self.q
        ncol = u.shape[1]
        U = u.reshape(n1, n1, n1, ncol)
        # 1/2 K u: z, then y passes shared by the three terms, then x
        az = _contract(self.A, U, 2, cnt)
        sz = _contract(self.S, U, 2, cnt)
        ayaz = _contract(self.A, az, 1, cnt)
        syaz = _contract(self.S, az, 1, cnt)
        aysz = _contract(self.A, sz, 1, cnt)
        t = syaz + aysz
        kin = _contract(self.S, ayaz, 0, cnt) + _contract(self.A, t, 0, cnt)
        if cnt is not None:
            cnt.flops += 2 * kin.size + kin.size          # the two sums and the 1/2
        kin = 0.5 * kin
        # V u: to the Gauss points, weight, back
        Uq = _contract(self.B, _contract(self.B, _contract(self.B, U, 2, cnt), 1, cnt), 0, cnt)
        Uq = Uq * (self.W * vq.reshape(q, q, q))[..., None]
        if cnt is not None:
            cnt.flops += Uq.size
        Bt = self.B.T
        pot = _contract(Bt, _contract(Bt, _contract(Bt, Uq, 0, cnt), 1, cnt), 2, cnt)
        if cnt is not None:
            cnt.flops += kin.size
        return (kin + pot).reshape(n1 ** 3, ncol)


def flops_per_cell(p: int, q: int | None = None) -> int:
    """Flops of MatrixFreeCell.apply per cell and vector (closed form of the count)."""
    n1 = p + 1
    q = q if q is not None else p + 2
    kinetic = 14 * n1 ** 4 + 3 * n1 ** 3
    potential = 4 * (q * n1 ** 3 + q * q * n1 * n1 + q ** 3 * n1) + q ** 3
    return kinetic + potential + n1 ** 3


def flops_dense_per_cell(p: int) -> int:
    """Dense cell product H_e u: 2 n_e^2 flops per cell and vector."""
    return 2 * (p + 1) ** 6


def apply_Htilde(prob, X: np.ndarray) -> np.ndarray:
    """H~ X = M^{-1/2} sum_e P_e^T H_e P_e M^{-1/2} X with every H_e applied
    matrix-free (local part only: the problem must have no projectors)."""
    if prob.C is not None:
        raise ValueError("matrix-free oracle covers the local Hamiltonian only")
    mesh, basis = prob.mesh, prob.basis
    cell = MatrixFreeCell(mesh.p, mesh.h, basis.q)
    Xs = prob.minv_sqrt[:, None] * np.asarray(X, dtype=np.float64)
    out = np.zeros_like(Xs)
    for e in range(mesh.ncells):
        d = mesh.cell_dofs(e)
        ok = d >= 0
        ue = np.zeros((mesh.ne, Xs.shape[1]))
        ue[ok] = Xs[d[ok]]
        vq = prob.potential(basis.quad_coords(mesh.cell_origin(e)))
        re = cell.apply(ue, vq)
        np.add.at(out, d[ok], re[ok])
    return prob.minv_sqrt[:, None] * out
