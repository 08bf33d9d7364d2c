"""Planted mistakes in the oracle must be caught by its pins.

Each case monkeypatches one plausible error into the oracle (on the CPU) and
checks that the corresponding closed-form pin no longer holds, so the pins
are shown to be sensitive to that class of mistake.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import chfsi, fe, hamiltonian as ham

FREE = 0.5 * (2 * np.pi / 10.0) ** 2


def _free_first_shell(prob):
    ev = np.linalg.eigvalsh(prob.dense_Htilde())
    return ev[1:7]


def test_dropped_half_in_kinetic_term_is_caught(monkeypatch):
    ok = ham.Problem(3, 4, 10.0, True, lambda x: np.zeros(len(x)))
    assert np.abs(_free_first_shell(ok) - FREE).max() < 2e-4 * FREE

    def bad(self, e):
        xq = self.basis.quad_coords(self.mesh.cell_origin(e))
        return self.K + self.basis.potential_matrix(self.potential(xq))
    monkeypatch.setattr(ham.Problem, "cell_hamiltonian", bad)
    wrong = ham.Problem(3, 4, 10.0, True, lambda x: np.zeros(len(x)))
    assert np.abs(_free_first_shell(wrong) - FREE).max() > 0.5 * FREE


def test_wrong_periodic_wrap_is_caught(monkeypatch):
    def bad_global(self, c, i, axis=0):
        g = c * self.p + i
        if self.per[axis]:
            return g if g < self.ncell * self.p else 1   # should wrap to 0
        return -1 if g in (0, self.ncell * self.p) else g - 1
    monkeypatch.setattr(fe.Mesh, "_global_1d", bad_global)
    wrong = ham.Problem(3, 4, 10.0, True, lambda x: np.zeros(len(x)))
    shell = _free_first_shell(wrong)
    assert np.abs(shell - FREE).max() > 1e-2 * FREE or shell.max() - shell.min() > 1e-6


def test_transposed_cholesky_factor_is_caught(monkeypatch):
    def bad(X):
        S = X.T @ X
        L = np.linalg.cholesky(S)
        Linv = sla.solve_triangular(L, np.eye(len(S)), lower=True)
        return X @ Linv              # should be L^{-T}
    monkeypatch.setattr(chfsi, "cholgs", bad)
    X = np.random.default_rng(3).uniform(-1, 1, (200, 12))
    Q = chfsi.cholgs(X)
    assert np.abs(Q.T @ Q - np.eye(12)).max() > 1e-3


def test_wrong_recurrence_sign_is_caught():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((60, 60))
    H = A + A.T
    evals, evecs = np.linalg.eigh(H)
    X = rng.standard_normal((60, 4))
    a, b, a0 = evals[10], evals[-1] * 1.01, evals[0]
    good = chfsi.chebyshev_filter(lambda Y: H @ Y, X, 6, a, b, a0)
    ref = chfsi.exact_filter(evals, evecs, X, 6, a, b, a0)
    assert np.linalg.norm(good - ref) < 1e-10 * np.linalg.norm(ref)
    # planted: + sigma_k sigma_{k+1} Y_{k-1} instead of minus
    e, c = (b - a) / 2, (b + a) / 2
    s1 = e / (a0 - c)
    s, Yp, Y = s1, X, (s1 / e) * (H @ X - c * X)
    for _ in range(2, 7):
        sn = 1 / (2 / s1 - s)
        Yp, Y, s = Y, (2 * sn / e) * (H @ Y - c * Y) + s * sn * Yp, sn
    assert np.linalg.norm(Y - ref) > 1e-3 * np.linalg.norm(ref)


def test_transposed_ritz_rotation_is_caught(monkeypatch):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((80, 80))
    H = A + A.T
    evals, evecs = np.linalg.eigh(H)
    V = evecs[:, :8] @ np.linalg.qr(rng.standard_normal((8, 8)))[0]

    def bad(apply_Ht, X):
        Hh = X.T @ apply_Ht(X)
        D, Q = np.linalg.eigh(0.5 * (Hh + Hh.T))
        return D, X @ Q.T            # should be X Q
    monkeypatch.setattr(chfsi, "rayleigh_ritz", bad)
    D, X = chfsi.rayleigh_ritz(lambda Y: H @ Y, V)
    R = np.linalg.norm(H @ X - X * D[None, :], axis=0)
    assert R.max() > 1e-3


def test_missing_mass_scaling_in_density_is_caught():
    """Density built from X~ instead of Psi = M^{-1/2} X~ breaks the uniform
    density of the constant state."""
    from oracle import density as od
    L = 4.0
    prob = ham.Problem(2, 3, L, True, lambda x: np.zeros(len(x)))
    x = np.sqrt(prob.mass) / np.sqrt(L ** 3)
    assert np.allclose(od.density(prob, x[:, None]), 2.0 / L ** 3, atol=1e-14)
    prob.minv_sqrt = np.ones_like(prob.minv_sqrt)          # planted: scaling dropped
    rho = od.density(prob, x[:, None])
    assert np.abs(rho - 2.0 / L ** 3).max() > 0.1 * 2.0 / L ** 3


def test_wrong_sign_of_fractional_correction_is_caught(monkeypatch):
    """(1 - f) instead of (f - 1) in Eq. elecDensSP breaks the identity with
    the fully rotated density."""
    from oracle import density as od
    from paper_1903_10959_gb300 import workloads as W
    s = W.small_periodic(seed=5, ncell=2, p=3, L=5.0, n_wells=3, n_want=12)
    prob = ham.wells_problem(s.ncell, s.p, s.L, True, s.centres, s.depths, s.widths)
    n, n_fr = 14, 5
    X = chfsi.cholgs(W.start_block(3, prob.ndofs, n))
    d_fr, X_fr = od.rayleigh_ritz_split(prob.apply_Htilde, X, n_fr)
    mu, occ = od.fermi_level(d_fr, n - n_fr, 2 * (n - n_fr) + 3.3, kT=0.05)
    D, XR = chfsi.rayleigh_ritz(prob.apply_Htilde, X)
    f = np.concatenate([np.ones(n - n_fr), occ])
    rho_full = od.density(prob, XR * np.sqrt(f)[None, :])
    rho_bad = od.density(prob, X, X_fr, 2.0 - occ)          # planted: f - 1 -> 1 - f
    assert np.abs(rho_bad - rho_full).max() > 1e-3 * np.abs(rho_full).max()


def test_periodic_images_along_a_dirichlet_axis_are_caught(monkeypatch):
    """Semi-periodic systems: a well summed over images along every axis,
    the Dirichlet one included, must fail the image pin."""
    monkeypatch.setattr(ham, "periodic_axes", lambda per: (True, True, True))
    c, d, w = np.array([[0.5, 0.5, 3.0]]), np.array([2.0]), np.array([1.0])
    b = np.array([[0.5, 0.5, 5.8]])
    v_slab = ham.gaussian_wells(b, c, d, w, 6.0, (True, True, False))[0]
    v_open = -2.0 * np.exp(-2.8 ** 2 / 2.0)          # the well itself; no z image
    assert abs(v_slab - v_open) > 1e-3


def test_dropped_k_squared_term_is_caught(monkeypatch):
    """Bloch Hamiltonian: without the 1/2 |k|^2 term the free-particle bands
    shift away from 1/2 |2 pi n / L + k|^2."""
    from oracle import kpoints as kp
    orig = kp.BlochProblem.__init__

    def bad(self, prob, k):
        orig(self, prob, k)
        kG = sum(self.k[d] * self.G[d] for d in range(3))
        self.shift = -1j * kG                        # 1/2 |k|^2 A dropped
    monkeypatch.setattr(kp.BlochProblem, "__init__", bad)
    L, k = 6.0, np.array([0.25, -0.4, 0.1])
    prob = ham.Problem(3, 4, L, True, lambda x: np.zeros(len(x)))
    ev = np.linalg.eigvalsh(kp.BlochProblem(prob, k).dense_Htilde())
    g = 2 * np.pi / L
    n = np.arange(-3, 4)
    G = np.stack(np.meshgrid(n, n, n, indexing="ij"), -1).reshape(-1, 3) * g
    ref = np.sort(0.5 * np.sum((G + k) ** 2, axis=1))
    assert not np.allclose(ev[:12], ref[:12], rtol=2e-3)


def test_dropped_four_pi_in_poisson_is_caught(monkeypatch):
    """SCF electrostatics: -(1/4 pi) lap phi = f solved without the 4 pi
    misses the single-Fourier-mode closed form."""
    from oracle import scf
    orig = scf.load_vector

    def bad(prob, fq):
        return orig(prob, fq) / (4.0 * np.pi)
    monkeypatch.setattr(scf, "load_vector", bad)
    L, amp = 6.0, 0.7
    prob = scf.FieldProblem(3, 4, L, True)
    xq = scf.gauss_points(prob)
    k = 2 * np.pi / L
    phi = scf.poisson_periodic(prob, amp * np.cos(k * xq[..., 0]))
    exact = 4 * np.pi * amp / k ** 2 * np.cos(k * prob.mesh.dof_coords()[:, 0])
    assert np.abs(phi - exact).max() > 0.5 * np.abs(exact).max()


def _mf_vs_dense_error():
    """Relative difference of the oracle's matrix-free apply and its dense
    cell-matrix apply (the pin of test_oracle_matrix_free.py) on a small
    periodic box with wells."""
    from oracle import matrix_free as mf
    rng = np.random.default_rng(2)
    c, d, w = rng.uniform(0, 5, (3, 3)), rng.uniform(1, 3, 3), rng.uniform(0.8, 1.2, 3)
    prob = ham.wells_problem(2, 5, 5.0, True, c, d, w)
    X = rng.uniform(-1, 1, (prob.ndofs, 4))
    ref = prob.apply_Htilde(X)
    return np.linalg.norm(mf.apply_Htilde(prob, X) - ref) / np.linalg.norm(ref)


def test_matrix_free_quadrature_weight_without_jacobian_is_caught(monkeypatch):
    from oracle import matrix_free as mf
    assert _mf_vs_dense_error() < 1e-13
    init = mf.MatrixFreeCell.__init__

    def bad(self, p, h, q=None):
        init(self, p, h, q)
        self.W = self.W / (h / 2.0) ** 3          # potential weights without jac^3
    monkeypatch.setattr(mf.MatrixFreeCell, "__init__", bad)
    assert _mf_vs_dense_error() > 1e-3


def test_matrix_free_mass_and_stiffness_factors_swapped_is_caught(monkeypatch):
    from oracle import matrix_free as mf
    init = mf.MatrixFreeCell.__init__

    def bad(self, p, h, q=None):
        init(self, p, h, q)
        self.A, self.S = self.S, self.A           # the 1-D factors in each other's place
    monkeypatch.setattr(mf.MatrixFreeCell, "__init__", bad)
    assert _mf_vs_dense_error() > 1e-3


def test_shared_wrong_exchange_constant_is_caught(monkeypatch):
    """Both LDA exchange functions with 3 / (2 pi) in place of 3 / pi stay
    consistent with each other (the derivative pin holds) but miss the
    uniform-gas constant."""
    from oracle import scf
    monkeypatch.setattr(scf, "lda_exchange_energy_density",
                        lambda rho: -0.75 * np.cbrt(3.0 * np.maximum(rho, 0.0) / (2 * np.pi)))
    monkeypatch.setattr(scf, "lda_exchange_potential",
                        lambda rho: -np.cbrt(3.0 * np.maximum(rho, 0.0) / (2 * np.pi)))
    rho = np.array([0.05, 0.4])
    h = 1e-6 * rho
    e = lambda r: r * scf.lda_exchange_energy_density(r)
    assert np.allclose(scf.lda_exchange_potential(rho), (e(rho + h) - e(rho - h)) / (2 * h), rtol=1e-7)
    rs = 1.0
    eps = scf.lda_exchange_energy_density(np.array([3.0 / (4.0 * np.pi * rs ** 3)]))[0] * rs
    assert abs(eps + 0.4581652932831429) > 1e-2
