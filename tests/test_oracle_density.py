"""Pins of the spectrum-splitting RR, Fermi level and density oracle
(Sec. 3.5, Algorithms rr and dc, Eq. elecDensSP) against closed forms,
exact polynomial reproduction and brute-force identities."""
import numpy as np
import pytest

from oracle import chfsi as och
from oracle import density as od
from oracle import hamiltonian as oh
from paper_1903_10959_gb300 import workloads as W


def _free(ncell=2, p=3, L=4.0, periodic=True):
    return oh.Problem(ncell, p, L, periodic, lambda x: np.zeros(len(x)))


def test_constant_state_gives_uniform_density():
    """Periodic free particle: the ground state is the constant 1/sqrt(V)
    (in the FE space exactly); one doubly occupied state gives rho = 2/V at
    every Gauss point."""
    L = 4.0
    prob = _free(L=L)
    x = np.sqrt(prob.mass) / np.sqrt(L ** 3)            # X~ = M^{1/2} Psi, Psi = 1/sqrt(V)
    assert abs(x @ x - 1.0) < 1e-13                      # GLL-mass normalised
    rho = od.density(prob, x[:, None])
    assert np.allclose(rho, 2.0 / L ** 3, rtol=0, atol=1e-14)


def test_polynomial_field_is_reproduced_at_gauss_points():
    """A Dirichlet field Psi = x(L-x) y(L-y) z(L-z) lies in the FE space (p >= 2):
    its density is 2 Psi(x_q)^2 exactly at every Gauss point."""
    L, p = 3.0, 3
    prob = oh.Problem(3, p, L, False, lambda x: np.zeros(len(x)))
    xyz = prob.mesh.dof_coords()
    f = lambda r: (r[:, 0] * (L - r[:, 0]) * r[:, 1] * (L - r[:, 1]) * r[:, 2] * (L - r[:, 2]))
    psi = f(xyz)
    x = np.sqrt(prob.mass) * psi                         # X~ = M^{1/2} Psi
    rho = od.density(prob, x[:, None])
    for e in [0, 7, 13, 26]:
        pts = prob.basis.quad_coords(prob.mesh.cell_origin(e))
        assert np.allclose(rho[e], 2.0 * f(pts) ** 2, rtol=1e-12, atol=1e-14)


def test_split_density_equals_full_rotation_density():
    """Eq. elecDensSP against its definition: 2 sum_i f_i |psi_i^R|^2 with the
    full rotation X Q and f_i = 1 below the partially occupied states."""
    s = W.small_periodic(seed=5, ncell=2, p=3, L=5.0, n_wells=3, n_want=12)
    prob = oh.wells_problem(s.ncell, s.p, s.L, True, s.centres, s.depths, s.widths)
    n, n_fr = 14, 5
    X = och.cholgs(W.start_block(3, prob.ndofs, n))
    d_fr, X_fr = od.rayleigh_ritz_split(prob.apply_Htilde, X, n_fr)
    mu, occ = od.fermi_level(d_fr, n - n_fr, 2 * (n - n_fr) + 3.3, kT=0.05)
    rho = od.density(prob, X, X_fr, occ)
    D, XR = och.rayleigh_ritz(prob.apply_Htilde, X)
    f = np.concatenate([np.ones(n - n_fr), occ])
    rho_full = od.density(prob, XR * np.sqrt(f)[None, :])
    assert np.allclose(rho, rho_full, rtol=1e-10, atol=1e-13)
    assert np.allclose(D[n - n_fr:], d_fr, atol=1e-12)


def test_split_rr_matches_full_rr_top_block():
    s = W.small_periodic(seed=6, ncell=2, p=3, L=5.0, n_wells=2, n_want=10)
    prob = oh.wells_problem(s.ncell, s.p, s.L, True, s.centres, s.depths, s.widths)
    X = och.cholgs(W.start_block(4, prob.ndofs, 12))
    D, XR = och.rayleigh_ritz(prob.apply_Htilde, X)
    d_fr, X_fr = od.rayleigh_ritz_split(prob.apply_Htilde, X, 4)
    assert np.allclose(d_fr, D[-4:], atol=1e-12)
    sign = np.sign((X_fr * XR[:, -4:]).sum(0))
    assert np.allclose(X_fr * sign, XR[:, -4:], atol=1e-10)


def test_fermi_level_closed_forms():
    # two states at 0 and 1 holding one pair of electrons: f(0) + f(1) = 1 iff mu = 1/2
    mu, occ = od.fermi_level([0.0, 1.0], 0, 2.0, kT=0.3)
    assert abs(mu - 0.5) < 1e-13 and abs(occ.sum() - 1.0) < 1e-13
    # a gap and a cold smearing: the lowest two of four states filled
    mu, occ = od.fermi_level([-1.0, -0.9, 0.9, 1.0], 3, 10.0, kT=0.01)
    assert -0.9 < mu < 0.9
    assert np.allclose(occ, [1, 1, 0, 0], atol=1e-30)
    # the constraint holds and the count grows with mu
    eps = np.linspace(-0.3, 0.4, 9)
    for ne in (20.5, 23.0, 27.9):
        mu, occ = od.fermi_level(eps, 6, ne, kT=0.05)
        assert abs(2 * (6 + occ.sum()) - ne) < 1e-12
    f1 = od.fermi_dirac(eps, 0.0, 0.05).sum()
    f2 = od.fermi_dirac(eps, 0.01, 0.05).sum()
    assert f2 > f1
    with pytest.raises(ValueError):
        od.fermi_level([0.0, 1.0], 0, 5.0, kT=0.1)


def test_density_integrates_to_electron_count_for_constant_occupations():
    """With f = 1 for all n states and M-orthonormal Psi, the Gauss-quadrature
    integral of rho is 2 sum_i Psi_i^T M_cons Psi_i = 2n up to the GLL mass
    lumping error, which vanishes for the constant state and stays small for
    smooth ones."""
    prob = _free(ncell=3, p=4, L=6.0)
    D = np.linalg.eigvalsh(prob.dense_Htilde())
    Ht = prob.dense_Htilde()
    w, V = np.linalg.eigh(Ht)
    X = V[:, :7]                                       # the lowest (smooth) states
    rho = od.density(prob, X)
    total = (rho * prob.basis.W[None, :]).sum()
    assert abs(total - 14.0) < 1e-3 * 14.0
    assert abs(D[0]) < 1e-10
