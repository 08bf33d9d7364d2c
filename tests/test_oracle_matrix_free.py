"""Pins of the matrix-free (sum-factorised) oracle apply: it reproduces the
dense cell-matrix apply of the same Hamiltonian (Eq. discreteHam; the two
differ only in the order of the sums), its 1-D factors rebuild the dense cell
matrices, and the flop count of the implementation equals its closed form."""
import numpy as np

from oracle import fe
from oracle import hamiltonian as oh
from oracle import matrix_free as mf


def test_one_dimensional_factors_rebuild_the_cell_matrices():
    p, h = 4, 1.7
    basis = fe.CellBasis(p, h)
    cell = mf.MatrixFreeCell(p, h)
    K = (np.kron(np.kron(cell.A, cell.A), cell.S) + np.kron(np.kron(cell.A, cell.S), cell.A)
         + np.kron(np.kron(cell.S, cell.A), cell.A))
    assert np.allclose(K, basis.stiffness(), rtol=0, atol=1e-12 * np.abs(K).max())
    rng = np.random.default_rng(1)
    vq = rng.uniform(-2, 1, basis.q ** 3)
    u = rng.standard_normal((basis.ne, 6))
    dense = (0.5 * basis.stiffness() + basis.potential_matrix(vq)) @ u
    assert np.allclose(cell.apply(u, vq), dense, rtol=0, atol=1e-12 * np.abs(dense).max())


def test_matrix_free_apply_equals_dense_apply():
    for periodic in (True, (True, False, True)):
        rng = np.random.default_rng(2)
        c, d, w = rng.uniform(0, 5, (3, 3)), rng.uniform(1, 3, 3), rng.uniform(0.8, 1.2, 3)
        prob = oh.wells_problem(2, 5, 5.0, periodic, c, d, w)
        X = rng.uniform(-1, 1, (prob.ndofs, 4))
        ref = prob.apply_Htilde(X)
        got = mf.apply_Htilde(prob, X)
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


def test_flop_count_matches_closed_form():
    for p in range(1, 9):
        cell = mf.MatrixFreeCell(p, 1.0)
        cnt = mf.Counter()
        cell.apply(np.ones(((p + 1) ** 3, 1)), np.ones(cell.q ** 3), cnt)
        assert cnt.flops == mf.flops_per_cell(p)
    # the dense product does more work from p = 4 on and grows as n1^6
    ratio = [mf.flops_dense_per_cell(p) / mf.flops_per_cell(p) for p in range(1, 9)]
    assert all(r < 1.0 for r in ratio[:3]) and all(r > 1.0 for r in ratio[3:])
    assert all(b > a for a, b in zip(ratio, ratio[1:]))
