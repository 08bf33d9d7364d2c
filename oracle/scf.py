"""Self-consistent field loop on Gaussian-charge systems (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Algorithm scf (Sec. 3.2) around the ChFSI step, in a periodic box:

* ES (step 4): the total electrostatic potential phi solves
      -(1 / 4 pi) lap phi = rho + b               (Eq. ksproblemPer)
  with the electron density rho >= 0 and the nuclear charge b < 0.  Reading:
  the nuclei are normalised Gaussians, b = -sum_I Z_I (2 pi s_I^2)^{-3/2}
  exp(-|x - R_I|^2 / (2 s_I^2)) over the periodic images, so no self-potential
  is needed.  FE form: K phi = 4 pi F, F_j = int N_j (rho + b) by the Gauss
  rule of the cells, with int phi = 0.  The discrete density carries the GLL
  lumping error of its normalisation, so its small net charge is neutralised
  by a uniform background (F_j -= Q int N_j / |box|).
* V_eff (step 5) = phi + V_x(rho), V_x = -(3 rho / pi)^{1/3}: the exchange
  part of the local-density approximation (reading: correlation omitted).
* Steps 6-7: cell Hamiltonians with V_eff at the Gauss points, then ChFSI
  passes (filter, CholGS, RR) warm-started from the previous step's block.
* DC (step 8): Fermi-Dirac occupations of all N states (the smearing of
  Sec. 3.2) and rho at the Gauss points (Eq. elecDensSP, every state
  partially occupied).
* Mixing (step 9, Sec. 3.6): n-stage Anderson mixing of rho (Anderson 1965).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from . import chfsi as och
from . import density as od
from .hamiltonian import Problem


class FieldProblem(Problem):
    """Problem whose V_eff is given by its values at the Gauss points of every
    cell, vq[e, a + q (b + q c)] (the layout of ``density.density``)."""

    def __init__(self, ncell, p, L, periodic=True, q=None):
        super().__init__(ncell, p, L, periodic, lambda x: np.zeros(len(x)), None, q)
        self.vq = np.zeros((self.mesh.ncells, self.basis.N.shape[0]))

    def set_vq(self, vq):
        """New V_eff at the Gauss points (step 5 of Algorithm scf); drops cached H_e."""
        self.vq = np.asarray(vq, dtype=np.float64).reshape(self.mesh.ncells, -1)
        self._cellH = {}

    def cell_hamiltonian(self, e: int) -> np.ndarray:
        """H_e = 1/2 K_e + V_e with V_e from the Gauss-point values (Eq. discreteHam)."""
        if e not in self._cellH:
            self._cellH[e] = 0.5 * self.K + self.basis.potential_matrix(self.vq[e])
        return self._cellH[e]


def gauss_points(prob) -> np.ndarray:
    """(ncells, q^3, 3) Gauss points of every cell."""
    return np.stack([prob.basis.quad_coords(prob.mesh.cell_origin(e)) for e in range(prob.mesh.ncells)])


def nuclear_charge(x, centres, Z, sigma, L):
    """b(x) = -sum_I Z_I g_I(x), normalised Gaussians of width sigma_I, periodic images."""
    x = np.asarray(x, dtype=np.float64)
    b = np.zeros(x.shape[:-1])
    for R, z, s in zip(np.asarray(centres), np.asarray(Z), np.asarray(sigma)):
        for sh in itertools.product((-1, 0, 1), repeat=3):
            d = x - (R + L * np.array(sh))
            b -= z * np.exp(-np.sum(d * d, axis=-1) / (2 * s * s)) / (2 * np.pi * s * s) ** 1.5
    return b


def assemble_stiffness(prob) -> sp.csr_matrix:
    """Global K_jl = int grad N_j . grad N_l (sparse)."""
    mesh, K = prob.mesh, prob.K
    rows, cols, vals = [], [], []
    for e in range(mesh.ncells):
        d = mesh.cell_dofs(e)
        ok = d >= 0
        dd = d[ok]
        rows.append(np.repeat(dd, len(dd)))
        cols.append(np.tile(dd, len(dd)))
        vals.append(K[np.ix_(ok, ok)].ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(mesh.ndofs, mesh.ndofs))
    A.sum_duplicates()
    return A


def load_vector(prob, fq) -> np.ndarray:
    """F_j = int N_j f for f given at the Gauss points (ncells, q^3)."""
    mesh, basis = prob.mesh, prob.basis
    F = np.zeros(mesh.ndofs)
    for e in range(mesh.ncells):
        d = mesh.cell_dofs(e)
        ok = d >= 0
        np.add.at(F, d[ok], (basis.N.T @ (basis.W * fq[e]))[ok])
    return F


def poisson_periodic(prob, fq, K=None) -> np.ndarray:
    """Nodal phi with -(1 / 4 pi) lap phi = f in the periodic box, int phi = 0;
    the net charge of f is neutralised by a uniform background."""
    if not prob.mesh.periodic:
        raise ValueError("periodic box only")
    K = assemble_stiffness(prob) if K is None else K
    F = load_vector(prob, fq)
    m = load_vector(prob, np.ones_like(fq))                  # int N_j
    F = F - F.sum() * m / m.sum()
    n = prob.mesh.ndofs
    A = sp.bmat([[K, sp.csr_matrix(m[:, None])], [sp.csr_matrix(m[None, :]), None]], format="csc")
    sol = spl.spsolve(A, np.concatenate([4.0 * np.pi * F, [0.0]]))
    return sol[:n]


def nodal_to_gauss(prob, u) -> np.ndarray:
    """Values of the FE field with nodal values u at the Gauss points (ncells, q^3)."""
    mesh, basis = prob.mesh, prob.basis
    out = np.zeros((mesh.ncells, basis.N.shape[0]))
    for e in range(mesh.ncells):
        d = mesh.cell_dofs(e)
        ok = d >= 0
        out[e] = basis.N[:, ok] @ u[d[ok]]
    return out


def lda_exchange_potential(rho):
    """Slater exchange V_x = d(rho eps_x)/d rho = -(3 rho / pi)^{1/3}."""
    return -np.cbrt(3.0 * np.maximum(rho, 0.0) / np.pi)


def lda_exchange_energy_density(rho):
    """eps_x = -(3/4) (3 rho / pi)^{1/3} (energy per electron)."""
    return -0.75 * np.cbrt(3.0 * np.maximum(rho, 0.0) / np.pi)


class Anderson:
    """n-stage Anderson mixing (Anderson 1965) for x = g(x): keeps the last
    ``depth`` pairs (x_i, r_i = g(x_i) - x_i), takes the affine combination of
    the pairs whose residual sum sum c_i r_i (sum c_i = 1) is smallest in the
    weighted norm, and returns sum c_i (x_i + beta r_i)."""

    def __init__(self, beta=0.5, depth=6, weights=None):
        self.beta, self.depth, self.w = beta, depth, weights
        self.xs, self.rs = [], []

    def step(self, x, gx):
        """Next iterate from the current x and g(x)."""
        x = np.asarray(x, dtype=np.float64).ravel()
        r = np.asarray(gx, dtype=np.float64).ravel() - x
        self.xs.append(x)
        self.rs.append(r)
        self.xs, self.rs = self.xs[-self.depth:], self.rs[-self.depth:]
        w = np.ones_like(r) if self.w is None else np.asarray(self.w).ravel()
        m = len(self.rs)
        if m == 1:
            c = np.ones(1)
        else:
            # minimise |r_m + sum_{i<m} t_i (r_i - r_m)|_w over t, c = (t, 1 - sum t)
            D = np.stack([self.rs[i] - self.rs[-1] for i in range(m - 1)], axis=1) * np.sqrt(w)[:, None]
            t, *_ = np.linalg.lstsq(D, -self.rs[-1] * np.sqrt(w), rcond=None)
            c = np.concatenate([t, [1.0 - t.sum()]])
        return sum(ci * (xi + self.beta * ri) for ci, xi, ri in zip(c, self.xs, self.rs))


def scf(ncell, p, L, centres, Z, sigma, n_states, kT=0.01, degree=20, passes=2, tol=1e-8,
        max_iter=60, beta=0.5, depth=6, seed=1):
    """Algorithm scf on a periodic Gaussian-charge system; returns a dict with
    the converged density at the Gauss points, the Ritz values, occupations,
    the nodal phi, the residual history and the problem."""
    prob = FieldProblem(ncell, p, L, True)
    xq = gauss_points(prob)
    bq = nuclear_charge(xq, centres, Z, sigma, L)
    n_el = float(np.sum(Z))
    W = prob.basis.W
    # initial density: the nuclear Gaussians widened to 1 bohr, scaled to n_el electrons
    rho = -nuclear_charge(xq, centres, Z, np.maximum(np.asarray(sigma), 1.0), L)
    rho *= n_el / np.sum(rho * W[None, :])
    K = assemble_stiffness(prob)
    rng = np.random.default_rng(seed)
    X = och.cholgs(rng.uniform(-1.0, 1.0, (prob.ndofs, n_states)))
    mixer = Anderson(beta=beta, depth=depth, weights=np.broadcast_to(W, rho.shape))
    hist = []
    for it in range(max_iter):
        phi = poisson_periodic(prob, rho + bq, K)                       # ES
        vq = nodal_to_gauss(prob, phi) + lda_exchange_potential(rho)    # V_eff
        prob.set_vq(vq)
        Ht = prob.apply_Htilde
        b_up = och.lanczos_upper_bound(Ht, rng.uniform(-1, 1, prob.ndofs), 20)
        D, X = och.rayleigh_ritz(Ht, X)
        for _ in range(passes):                                          # ChFSI
            X = och.chebyshev_filter(Ht, X, degree, D[-1], b_up, D[0])
            X = och.cholgs(X)
            D, X = och.rayleigh_ritz(Ht, X)
        mu, occ = od.fermi_level(D, 0, n_el, kT)                         # DC
        rho_out = od.density(prob, X * np.sqrt(occ)[None, :])
        res = float(np.sqrt(np.sum(W[None, :] * (rho_out - rho) ** 2)))
        hist.append(res)
        if res < tol:
            rho = rho_out
            break
        rho = mixer.step(rho, rho_out).reshape(rho.shape)                # mixing
    return dict(rho=rho, evals=D, occ=occ, mu=mu, phi=phi, vq=vq, X=X, residuals=hist,
                problem=prob, bq=bq)
