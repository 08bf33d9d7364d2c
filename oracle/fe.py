"""Spectral finite elements on a uniform hexahedral mesh (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows Sec. 2.4 of arXiv:1903.10959: wavefunctions are expanded in C0
Lagrange polynomials interpolated over Gauss-Lobatto-Legendre (GLL) nodes
(Eq. fem); the local Hamiltonian entries are 1/2 int grad N_j . grad N_k +
int V N_j N_k (Eq. discreteHam); the overlap ("mass") matrix is evaluated
with GLL quadrature, which makes it diagonal (text after Eq. hep).  The
paper does not fix the quadrature of the Hamiltonian integrals; this oracle
uses a Gauss-Legendre rule with q = p + 2 points per direction, which is
exact for the stiffness on an affine cube and for the potential term when V
is a polynomial of degree <= 2.

Everything is written as the plain quadrature sums over the q^3 points of a
cell, with no tensor-product factorisation.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def gll_rule(p: int):
    """GLL nodes and weights on [-1, 1] with p + 1 points.

    Nodes: the end points and the roots of P_p'; weights
    w_i = 2 / (p (p + 1) P_p(x_i)^2) (Sec. 2.4: spectral basis on GLL points).
    """
    if p < 1:
        raise ValueError("p >= 1 required")
    c = np.zeros(p + 1)
    c[p] = 1.0
    dc = npleg.legder(c)
    ddc = npleg.legder(dc)
    inner = np.sort(npleg.legroots(dc).real) if p >= 2 else np.zeros(0)
    for _ in range(3):  # Newton polish of the roots of P_p'
        inner = inner - npleg.legval(inner, dc) / npleg.legval(inner, ddc)
    x = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (p * (p + 1) * npleg.legval(x, c) ** 2)
    return x, w


def gauss_rule(q: int):
    """Gauss-Legendre nodes and weights on [-1, 1] (q points, exact to 2q-1)."""
    return npleg.leggauss(q)


def lagrange_values(nodes: np.ndarray, t: np.ndarray) -> np.ndarray:
    """l_j(t_a) for the Lagrange polynomials on ``nodes``; shape (len(t), len(nodes))."""
    t = np.asarray(t, dtype=np.float64)
    n = len(nodes)
    out = np.ones((len(t), n))
    for j in range(n):
        for k in range(n):
            if k != j:
                out[:, j] *= (t - nodes[k]) / (nodes[j] - nodes[k])
    return out


def lagrange_derivs(nodes: np.ndarray, t: np.ndarray) -> np.ndarray:
    """l_j'(t_a) by the product rule: sum over the dropped factor m."""
    t = np.asarray(t, dtype=np.float64)
    n = len(nodes)
    out = np.zeros((len(t), n))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            term = np.full(len(t), 1.0 / (nodes[j] - nodes[m]))
            for k in range(n):
                if k != j and k != m:
                    term *= (t - nodes[k]) / (nodes[j] - nodes[k])
            out[:, j] += term
    return out


def local_index(p: int, i: int, j: int, k: int) -> int:
    """Local node number within a cell: x index fastest."""
    return i + (p + 1) * (j + (p + 1) * k)


class CellBasis:
    """3-D tensor-product basis N_{ijk} = l_i(x) l_j(y) l_k(z) on a cube of side h,
    tabulated at the q^3 Gauss points (Eq. fem, Eq. discreteHam)."""

    def __init__(self, p: int, h: float, q: int | None = None):
        self.p, self.h = p, h
        self.q = q if q is not None else p + 2
        self.nodes, self.gll_w = gll_rule(p)
        self.xq, self.wq = gauss_rule(self.q)
        n1 = p + 1
        self.ne = n1 ** 3
        v = lagrange_values(self.nodes, self.xq)     # (q, p+1)
        d = lagrange_derivs(self.nodes, self.xq)     # (q, p+1) d/dxi
        q = self.q
        nq = q ** 3
        self.N = np.zeros((nq, self.ne))
        self.dN = np.zeros((nq, self.ne, 3))
        self.W = np.zeros(nq)
        self.ref_pts = np.zeros((nq, 3))             # reference coords in [-1,1]^3
        jac = h / 2.0
        for c in range(q):
            for b in range(q):
                for a in range(q):
                    qi = a + q * (b + q * c)
                    self.W[qi] = self.wq[a] * self.wq[b] * self.wq[c] * jac ** 3
                    self.ref_pts[qi] = (self.xq[a], self.xq[b], self.xq[c])
                    for k in range(n1):
                        for j in range(n1):
                            for i in range(n1):
                                n = local_index(p, i, j, k)
                                self.N[qi, n] = v[a, i] * v[b, j] * v[c, k]
                                self.dN[qi, n, 0] = d[a, i] * v[b, j] * v[c, k] / jac
                                self.dN[qi, n, 1] = v[a, i] * d[b, j] * v[c, k] / jac
                                self.dN[qi, n, 2] = v[a, i] * v[b, j] * d[c, k] / jac

    def stiffness(self) -> np.ndarray:
        """K_jk = int grad N_j . grad N_k (Eq. discreteHam, first term without 1/2)."""
        return np.einsum("q,qjd,qkd->jk", self.W, self.dN, self.dN)

    def potential_matrix(self, vq: np.ndarray) -> np.ndarray:
        """V_jk = int V N_j N_k with V given at the q^3 Gauss points (Eq. discreteHam):
        sum over the points q of W_q V_q N_j(q) N_k(q)."""
        return self.N.T @ ((self.W * vq)[:, None] * self.N)

    def gll_mass_diag(self) -> np.ndarray:
        """Cell mass by GLL quadrature at the element nodes: N_j(x_k) = delta_jk,
        so M_e = diag(w_i w_j w_k (h/2)^3) (text after Eq. hep)."""
        n1 = self.p + 1
        jac = self.h / 2.0
        gv = lagrange_values(self.nodes, self.nodes)  # identity up to rounding
        out = np.zeros(self.ne)
        for k in range(n1):
            for j in range(n1):
                for i in range(n1):
                    w = self.gll_w[i] * self.gll_w[j] * self.gll_w[k] * jac ** 3
                    # sum_pts w_pt N_n(pt)^2 where pt runs over the GLL points
                    for kk in range(n1):
                        for jj in range(n1):
                            for ii in range(n1):
                                n = local_index(self.p, ii, jj, kk)
                                out[n] += w * (gv[i, ii] * gv[j, jj] * gv[k, kk]) ** 2
        return out

    def node_coords(self, cell_origin: np.ndarray) -> np.ndarray:
        """Physical coordinates of the cell's GLL nodes, shape (ne, 3)."""
        n1 = self.p + 1
        out = np.zeros((self.ne, 3))
        for k in range(n1):
            for j in range(n1):
                for i in range(n1):
                    n = local_index(self.p, i, j, k)
                    out[n] = cell_origin + (np.array([self.nodes[i], self.nodes[j],
                                                      self.nodes[k]]) + 1.0) * self.h / 2.0
        return out

    def quad_coords(self, cell_origin: np.ndarray) -> np.ndarray:
        """Physical coordinates of the q^3 Gauss points of the cell."""
        return cell_origin[None, :] + (self.ref_pts + 1.0) * self.h / 2.0


def periodic_axes(periodic) -> tuple:
    """Per-axis periodicity (x, y, z) from one flag for all axes or three flags."""
    if np.ndim(periodic) == 0:
        return (bool(periodic),) * 3
    t = tuple(bool(v) for v in periodic)
    if len(t) != 3:
        raise ValueError("periodic: one flag or three (x, y, z)")
    return t


class Mesh:
    """Uniform mesh of ncell^3 cubes of side h = L / ncell on [0, L]^3.

    Each axis is periodic or Dirichlet (periodic, non-periodic and
    semi-periodic boundary conditions, Sec. 1 and Sec. 2.1-2.2).  Periodic
    axis: global node g = (c p + i) mod (ncell p), so the nodes of opposite
    faces are identified.  Dirichlet axis: homogeneous Dirichlet, the boundary
    nodes g = 0 and g = ncell p are removed from the unknowns (H^1_0 along
    that axis).  Unknowns are numbered x fastest.
    """

    def __init__(self, ncell: int, p: int, L: float, periodic):
        self.ncell, self.p, self.L = ncell, p, L
        self.per = periodic_axes(periodic)
        self.periodic = all(self.per)
        self.h = L / ncell
        self.nd = tuple(ncell * p if pa else ncell * p - 1 for pa in self.per)
        self.ndofs = self.nd[0] * self.nd[1] * self.nd[2]
        self.ncells = ncell ** 3
        self.ne = (p + 1) ** 3

    def cell_coords(self, e: int):
        """(cx, cy, cz) of cell e, x fastest."""
        n = self.ncell
        return e % n, (e // n) % n, e // (n * n)

    def cell_origin(self, e: int) -> np.ndarray:
        """Lower corner of cell e (cells of side h on the uniform mesh, Sec. 3.1)."""
        cx, cy, cz = self.cell_coords(e)
        return np.array([cx, cy, cz], dtype=np.float64) * self.h

    def _global_1d(self, c: int, i: int, axis: int = 0) -> int:
        g = c * self.p + i
        if self.per[axis]:
            return g % (self.ncell * self.p)
        if g == 0 or g == self.ncell * self.p:
            return -1
        return g - 1

    def cell_dofs(self, e: int) -> np.ndarray:
        """Global unknown of each local node of cell e (-1: eliminated node)."""
        cx, cy, cz = self.cell_coords(e)
        p = self.p
        nx, ny = self.nd[0], self.nd[1]
        out = np.empty(self.ne, dtype=np.int64)
        for k in range(p + 1):
            gz = self._global_1d(cz, k, 2)
            for j in range(p + 1):
                gy = self._global_1d(cy, j, 1)
                for i in range(p + 1):
                    gx = self._global_1d(cx, i, 0)
                    n = local_index(p, i, j, k)
                    if gx < 0 or gy < 0 or gz < 0:
                        out[n] = -1
                    else:
                        out[n] = gx + nx * (gy + ny * gz)
        return out

    def dofmap(self) -> np.ndarray:
        """cell_dofs for every cell, shape (ncells, ne) (same rule, vectorised)."""
        n, p = self.ncell, self.p
        e = np.arange(self.ncells)
        c = np.stack([e % n, (e // n) % n, e // (n * n)], axis=1)
        i = np.arange(p + 1)
        g = c[:, :, None] * p + i[None, None, :]           # (ncells, 3, p+1)
        for a in range(3):
            if self.per[a]:
                g[:, a] = g[:, a] % (n * p)
            else:
                g[:, a] = np.where((g[:, a] == 0) | (g[:, a] == n * p), -1, g[:, a] - 1)
        gx = g[:, 0][:, None, None, :]
        gy = g[:, 1][:, None, :, None]
        gz = g[:, 2][:, :, None, None]
        d = gx + self.nd[0] * (gy + self.nd[1] * gz)
        bad = (gx < 0) | (gy < 0) | (gz < 0)
        return np.where(bad, -1, d).reshape(self.ncells, -1)

    def dof_coords(self) -> np.ndarray:
        """Physical coordinates of the unknowns (periodic nodes in [0, L))."""
        nodes, _ = gll_rule(self.p)
        x1 = []
        for a in range(3):
            g = np.arange(self.nd[a]) if self.per[a] else np.arange(1, self.nd[a] + 1)
            x1.append((g // self.p) * self.h + (nodes[g % self.p] + 1.0) * self.h / 2.0)
        X, Y, Z = np.meshgrid(x1[0], x1[1], x1[2], indexing="ij")
        return np.stack([X.T.ravel(), Y.T.ravel(), Z.T.ravel()], axis=1)


def assemble_mass_diag(mesh: Mesh, basis: CellBasis) -> np.ndarray:
    """Global diagonal M_jj = sum over cells of the GLL cell mass (text after Eq. hep)."""
    me = basis.gll_mass_diag()
    M = np.zeros(mesh.ndofs)
    for e in range(mesh.ncells):
        d = mesh.cell_dofs(e)
        ok = d >= 0
        np.add.at(M, d[ok], me[ok])
    return M
