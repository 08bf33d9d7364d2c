"""Pins of the oracle's Hamiltonian against physics with closed-form answers."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle import hamiltonian as ham

L = 10.0
FREE = 0.5 * (2 * np.pi / L) ** 2     # 1/2 (2 pi / L)^2


def _free(n, p):
    return ham.Problem(n, p, L, True, lambda x: np.zeros(len(x)))


def test_htilde_symmetric_with_wells_and_projectors():
    rng = np.random.default_rng(0)
    c = rng.uniform(0, 6, (3, 3))
    prob = ham.wells_problem(2, 3, 6.0, True, c, [1.0, 2.0, 1.5], [1.0, 0.9, 1.1],
                             projectors=dict(centres=c[:2], sigma=0.8, rcut=2.0,
                                             h=[[1, 0.5, 0.7, 2.0], [0.6, 1.2, 1.0, 1.9]]))
    H = prob.dense_Htilde()
    assert np.abs(H - H.T).max() <= 1e-15 * np.abs(H).max() * 10
    # the operator form agrees with the assembled matrix
    X = rng.standard_normal((prob.ndofs, 3))
    assert np.abs(prob.apply_Htilde(X) - H @ X).max() < 1e-12 * np.abs(H).max()
    S = prob.sparse_Htilde()
    assert np.abs(S.toarray() - H).max() < 1e-13 * np.abs(H).max()


def test_free_particle_spectrum_and_multiplicities():
    ev = np.linalg.eigvalsh(_free(3, 4).dense_Htilde())
    assert abs(ev[0]) < 1e-12
    # shells |n|^2 = 1, 2, 3 with multiplicities 6, 12, 8
    shells = [(1, 6), (2, 12), (3, 8)]
    i = 1
    for n2, mult in shells:
        grp = ev[i:i + mult]
        assert grp.max() - grp.min() < 1e-10                 # cubic symmetry: exact degeneracy
        assert abs(grp.mean() - n2 * FREE) < 2e-4 * n2 * FREE  # FE error at h = 10/3, p = 4
        i += mult
    assert ev[i] - ev[i - 1] > 1e-3                            # next shell starts after 27 states


def test_free_particle_converges_at_rate_2p():
    errs = []
    for n in (3, 4):
        ev = np.linalg.eigvalsh(_free(n, 2).dense_Htilde())
        errs.append(abs(ev[1] - FREE))
    slope = np.log(errs[0] / errs[1]) / np.log(4 / 3)
    assert 3.5 < slope < 5.0          # O(h^{2p}) with p = 2
    # higher degree is more accurate at the same number of unknowns per side
    e3 = abs(np.linalg.eigvalsh(_free(3, 3).dense_Htilde())[1] - FREE)
    e4 = abs(np.linalg.eigvalsh(_free(2, 4).dense_Htilde())[1] - FREE)
    assert e3 < errs[1] * 0.1 and e4 < errs[0]


@pytest.mark.slow
def test_harmonic_oscillator_levels():
    prob = ham.Problem(4, 6, 12.0, False, lambda x: ham.harmonic(x, [6, 6, 6], 1.0))
    ev = np.sort(spl.eigsh(prob.sparse_Htilde(), k=10, sigma=0.0, which="LM")[0])
    assert abs(ev[0] - 1.5) < 1e-4
    assert np.abs(ev[1:4] - 2.5).max() < 1e-4 and ev[3] - ev[1] < 1e-10
    assert np.abs(ev[4:10] - 3.5).max() < 2e-3


def test_projector_integrals_closed_form():
    sigma = 0.8
    c = np.array([5.0, 5.0, 5.0])       # box centre: the mesh is symmetric about it
    prob = ham.Problem(5, 5, 10.0, True, lambda x: np.zeros(len(x)),
                       projectors=dict(centres=c[None, :], sigma=sigma, rcut=100.0,
                                       h=[[1.0, 1.0, 1.0, 1.0]]))
    C = prob.C.toarray()
    G = (2 * np.pi * sigma ** 2) ** 1.5
    X = prob.mesh.dof_coords()
    # partition of unity: sum_j C_{k,j} = int chi_k
    assert abs(C[0].sum() - G) < 1e-8 * G
    assert np.abs(C[1:].sum(1)).max() < 1e-13
    # linear reproduction: sum_j C_{px,j} x_j = int chi_px x = sigma G (up to the
    # Gauss-rule error of the smooth integrand g (x - c) x)
    assert abs(C[1] @ X[:, 0] - sigma * G) < 1e-4 * G
    assert abs(C[2] @ X[:, 1] - sigma * G) < 1e-4 * G
    assert abs(C[3] @ X[:, 2] - sigma * G) < 1e-4 * G
    assert abs(C[1] @ X[:, 1]) < 1e-12 * G
    # H^nl = C^T h C with h > 0 is PSD of rank 4: its nonzero spectrum is that of
    # h^{1/2} C C^T h^{1/2}, and the four channels are linearly independent
    ev = np.linalg.eigvalsh(C @ C.T)
    assert ev.min() > 1e-6 * ev.max()
    X0 = np.random.default_rng(0).standard_normal((prob.ndofs, 3))
    q = np.einsum("ij,ij->j", X0, prob.apply_H(X0))
    assert np.all(q >= -1e-12 * np.abs(q).max())


def test_gaussian_wells_periodic_images():
    x = np.array([[0.1, 0.1, 0.1], [9.9, 9.9, 9.9]])
    v = ham.gaussian_wells(x, [[0.0, 0.0, 0.0]], [2.0], [1.0], 10.0, True)
    assert abs(v[0] - v[1]) < 1e-14          # symmetric about the periodic origin
    assert abs(v[0] + 2.0 * np.exp(-0.03 / 2)) < 1e-12
    v_np = ham.gaussian_wells(x, [[0.0, 0.0, 0.0]], [2.0], [1.0], 10.0, False)
    assert abs(v_np[1]) < 1e-30


def test_sampled_rows_match_full_apply():
    rng = np.random.default_rng(2)
    c = rng.uniform(0, 6, (2, 3))
    for periodic in (True, False):
        prob = ham.wells_problem(3, 2, 6.0, periodic, c, [1.0, 2.0], [1.0, 0.9],
                                 projectors=dict(centres=c[:1], sigma=0.8, rcut=2.0,
                                                 h=[[1, 0.5, 0.7, 2.0]]))
        X = rng.standard_normal((prob.ndofs, 4))
        rows = rng.choice(prob.ndofs, 9, replace=False)
        full = prob.apply_Htilde(X)
        assert np.abs(prob.apply_Htilde_rows(rows, X) - full[rows]).max() < 1e-12 * np.abs(full).max()
