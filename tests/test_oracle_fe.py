"""Pins of the oracle's finite-element layer (Sec. 2.4) against closed forms."""
import math
import os

import numpy as np
import pytest

from oracle import fe

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")


def _golden_gll():
    rows = {}
    env = {"sqrt": math.sqrt}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p, x, w = line.split()
            rows.setdefault(int(p), []).append((eval(x, env), eval(w, env)))
    return rows


def test_gll_matches_closed_forms():
    for p, pts in _golden_gll().items():
        x, w = fe.gll_rule(p)
        xr = np.array([a for a, _ in pts])
        wr = np.array([b for _, b in pts])
        assert np.allclose(x, xr, rtol=0, atol=1e-15)
        assert np.allclose(w, wr, rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_gll_exact_to_degree_2p_minus_1(p):
    x, w = fe.gll_rule(p)
    for k in range(2 * p):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    # and not beyond: degree 2p is integrated with an error
    assert abs(np.dot(w, x ** (2 * p)) - 2.0 / (2 * p + 1)) > 1e-6


@pytest.mark.parametrize("q", [2, 5, 9])
def test_gauss_exact_to_degree_2q_minus_1(q):
    x, w = fe.gauss_rule(q)
    for k in range(2 * q):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("p", [1, 3, 6, 7])
def test_lagrange_cardinality_partition_and_derivative(p):
    nodes, _ = fe.gll_rule(p)
    V = fe.lagrange_values(nodes, nodes)
    assert np.allclose(V, np.eye(p + 1), atol=1e-14)
    t = np.linspace(-1, 1, 37)
    assert np.allclose(fe.lagrange_values(nodes, t).sum(1), 1.0, atol=1e-13)
    d = fe.lagrange_derivs(nodes, t)
    assert np.allclose(d.sum(1), 0.0, atol=1e-11)
    hstep = 1e-6
    fd = (fe.lagrange_values(nodes, t + hstep) - fe.lagrange_values(nodes, t - hstep)) / (2 * hstep)
    assert np.allclose(d, fd, atol=1e-6 * max(1.0, np.abs(d).max()))
    # derivative of the interpolant of t^p is p t^(p-1) exactly
    assert np.allclose(d @ nodes ** p, p * t ** (p - 1), atol=1e-11)


@pytest.mark.parametrize("p", [2, 4])
def test_stiffness_nullspace_symmetry_and_energy(p):
    h = 1.7
    B = fe.CellBasis(p, h)
    K = B.stiffness()
    assert np.allclose(K, K.T, atol=1e-14 * np.abs(K).max())
    assert np.abs(K @ np.ones(B.ne)).max() < 1e-12 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert abs(ev[0]) < 1e-12 * ev[-1] and ev[1] > 1e-6
    # u = x^2 y + z lies in Q_p for p >= 2: u^T K u = int |grad u|^2 over [0, h]^3
    xyz = B.node_coords(np.zeros(3))
    u = xyz[:, 0] ** 2 * xyz[:, 1] + xyz[:, 2]
    exact = 4 * h ** 7 / 9 + h ** 7 / 5 + h ** 3
    assert abs(u @ K @ u - exact) < 1e-12 * exact


@pytest.mark.parametrize("p", [3, 5])
def test_gll_cell_mass_integrates_polynomials(p):
    h = 0.9
    B = fe.CellBasis(p, h)
    m = B.gll_mass_diag()
    xyz = B.node_coords(np.array([0.3, -0.2, 1.0]))
    assert abs(m.sum() - h ** 3) < 1e-14
    # x^a y^b z^c with a, b, c <= 2p - 1 integrated exactly by the GLL rule
    for a, b, c in [(2 * p - 1, 0, 1), (1, 2 * p - 1, 2), (p, p, 2 * p - 1)]:
        f = xyz[:, 0] ** a * xyz[:, 1] ** b * xyz[:, 2] ** c
        def I(k, lo):
            return ((lo + h) ** (k + 1) - lo ** (k + 1)) / (k + 1)
        exact = I(a, 0.3) * I(b, -0.2) * I(c, 1.0)
        assert abs(m @ f - exact) < 1e-12 * max(1.0, abs(exact))


def test_potential_matrix_constant_and_linear():
    p, h = 3, 1.3
    B = fe.CellBasis(p, h)
    one = np.ones(B.ne)
    xq = B.quad_coords(np.zeros(3))
    V = B.potential_matrix(np.full(len(xq), 2.5))
    assert abs(one @ V @ one - 2.5 * h ** 3) < 1e-13
    V = B.potential_matrix(xq[:, 0])
    assert abs(one @ V @ one - h ** 4 / 2) < 1e-13
    # quadratic V * (degree-p u)^2 is exact with q = p + 2: V = x^2, u = y
    xyz = B.node_coords(np.zeros(3))
    V = B.potential_matrix(xq[:, 0] ** 2)
    u = xyz[:, 1]
    assert abs(u @ V @ u - (h ** 3 / 3) * (h ** 3 / 3) * h) < 1e-13


@pytest.mark.parametrize("periodic", [True, False])
def test_dofmap_covers_unknowns(periodic):
    mesh = fe.Mesh(3, 2, 6.0, periodic)
    dm = mesh.dofmap()
    assert dm.shape == (27, 27)
    assert np.array_equal(dm, np.stack([mesh.cell_dofs(e) for e in range(27)]))
    used = dm[dm >= 0]
    assert set(used.tolist()) == set(range(mesh.ndofs))
    counts = np.bincount(used, minlength=mesh.ndofs)
    if periodic:
        assert mesh.ndofs == 6 ** 3
        # node multiplicities 1 (cell interior), 2 (face), 4 (edge), 8 (vertex)
        assert set(np.unique(counts).tolist()) == {1, 2, 4, 8}
        assert np.sum(counts == 8) == 27
    else:
        assert mesh.ndofs == 5 ** 3
        assert np.sum(dm < 0) > 0
    # coordinates agree with the cell-local node coordinates
    B = fe.CellBasis(2, mesh.h)
    X = mesh.dof_coords()
    for e in [0, 13, 26]:
        d = dm[e]
        ok = d >= 0
        xc = B.node_coords(mesh.cell_origin(e))[ok]
        diff = X[d[ok]] - xc
        if periodic:
            diff = diff - mesh.L * np.round(diff / mesh.L)
        assert np.abs(diff).max() < 1e-13


def test_global_mass_sums_to_volume():
    mesh = fe.Mesh(3, 4, 7.0, True)
    B = fe.CellBasis(4, mesh.h)
    M = fe.assemble_mass_diag(mesh, B)
    assert abs(M.sum() - 7.0 ** 3) < 1e-11
    assert M.min() > 0
