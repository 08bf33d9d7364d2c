"""Pins of the oracle's per-axis boundary conditions (periodic, non-periodic
and semi-periodic systems, Sec. 1 and Sec. 2.1-2.2): the all-periodic and
all-Dirichlet flags, the free-particle slab against its closed-form levels,
and the slab's z-only modes against an independent 1-D FE problem."""
import numpy as np
import scipy.linalg as sla

from oracle import fe
from oracle import hamiltonian as oh


def _zero(x):
    return np.zeros(len(x))


def test_three_flags_equal_one_flag():
    for flag in (True, False):
        a = fe.Mesh(3, 3, 6.0, flag)
        b = fe.Mesh(3, 3, 6.0, (flag,) * 3)
        assert a.ndofs == b.ndofs
        assert np.array_equal(a.dofmap(), b.dofmap())
        assert np.array_equal(a.dof_coords(), b.dof_coords())
    rng = np.random.default_rng(0)
    c, d, w = rng.uniform(0, 6, (3, 3)), rng.uniform(1, 3, 3), rng.uniform(0.8, 1.2, 3)
    pa = oh.wells_problem(2, 3, 6.0, True, c, d, w)
    pb = oh.wells_problem(2, 3, 6.0, (True, True, True), c, d, w)
    X = rng.uniform(-1, 1, (pa.ndofs, 3))
    assert np.abs(pa.apply_Htilde(X) - pb.apply_Htilde(X)).max() == 0.0


def test_slab_dof_layout():
    m = fe.Mesh(3, 2, 6.0, (True, False, True))
    assert m.nd == (6, 5, 6) and m.ndofs == 180
    dm = m.dofmap()
    used = np.unique(dm[dm >= 0])
    assert np.array_equal(used, np.arange(m.ndofs))       # every unknown appears
    xyz = m.dof_coords()
    assert xyz[:, 1].min() > 0 and xyz[:, 1].max() < 6.0   # Dirichlet faces y = 0, L removed
    assert xyz[:, 0].min() == 0.0                          # periodic x keeps x = 0 (x = L identified)
    for e in (0, 5, 26):                                   # the cell's own nodes map to their coordinates
        d = m.cell_dofs(e)
        ok = d >= 0
        o = m.cell_origin(e)
        nodes, _ = fe.gll_rule(2)
        loc = np.array([[o[0] + (nodes[i] + 1) * 1.0, o[1] + (nodes[j] + 1) * 1.0, o[2] + (nodes[k] + 1) * 1.0]
                        for k in range(3) for j in range(3) for i in range(3)])
        got = xyz[d[ok]]
        want = np.mod(loc[ok], 6.0)
        want[:, 1] = loc[ok][:, 1]
        assert np.allclose(got, want, atol=1e-12)


def _levels_slab(L, nmax=3):
    """Continuum free-particle levels, periodic x, y and Dirichlet z on [0, L]^3."""
    k, kz = 2 * np.pi / L, np.pi / L
    ev = [0.5 * (k * k * (a * a + b * b) + kz * kz * c * c)
          for a in range(-nmax, nmax + 1) for b in range(-nmax, nmax + 1) for c in range(1, nmax + 2)]
    return np.sort(ev)


def _fe_1d_dirichlet(ncell, p, L):
    """Generalised eigenvalues of (1/2 S, M) for the 1-D Dirichlet problem on
    [0, L]: stiffness by exact Gauss quadrature of the Lagrange derivatives on
    the GLL nodes (barycentric formula, written here), lumped GLL mass."""
    nodes, weights = fe.gll_rule(p)
    xg, wg = np.polynomial.legendre.leggauss(p + 2)
    # barycentric weights and derivatives of the Lagrange basis at the Gauss points
    bw = np.array([1.0 / np.prod([nodes[i] - nodes[j] for j in range(p + 1) if j != i])
                   for i in range(p + 1)])
    dl = np.zeros((len(xg), p + 1))
    for q, t in enumerate(xg):
        for i in range(p + 1):
            s = 0.0
            for m in range(p + 1):
                if m == i:
                    continue
                prod = 1.0
                for j in range(p + 1):
                    if j not in (i, m):
                        prod *= t - nodes[j]
                s += prod
            dl[q, i] = s * bw[i]
    h = L / ncell
    Se = (dl * wg[:, None]).T @ dl * (2.0 / h)
    n = ncell * p + 1
    S = np.zeros((n, n))
    M = np.zeros(n)
    for c in range(ncell):
        idx = np.arange(c * p, c * p + p + 1)
        S[np.ix_(idx, idx)] += Se
        M[idx] += weights * h / 2.0
    S, M = S[1:-1, 1:-1], M[1:-1]
    return sla.eigh(0.5 * S, np.diag(M), eigvals_only=True)


def test_slab_free_particle_levels():
    L, ncell, p = 6.0, 3, 4
    prob = oh.Problem(ncell, p, L, (True, True, False), _zero)
    ev = np.linalg.eigvalsh(prob.dense_Htilde())
    ref = _levels_slab(L)
    assert np.allclose(ev[:6], ref[:6], rtol=2e-3)
    # (0,0,1), (0,0,2), then the fourfold (+-1,0,1), (0,+-1,1) shell
    assert abs(ev[2] - ev[5]) < 1e-10 and ev[6] - ev[5] > 1e-3
    # modes constant along the periodic axes reduce exactly to the 1-D
    # Dirichlet problem (the GLL-lumped mass equals the consistent mass times
    # a constant), so those levels match the independent 1-D FE solution
    e1 = _fe_1d_dirichlet(ncell, p, L)
    assert abs(ev[0] - e1[0]) < 1e-12 and abs(ev[1] - e1[1]) < 1e-12


def test_slab_wells_are_periodic_only_along_periodic_axes():
    L = 6.0
    c, d, w = np.array([[0.5, 0.5, 3.0]]), np.array([2.0]), np.array([1.0])
    gw = lambda x, per: oh.gaussian_wells(np.array([x]), c, d, w, L, per)[0]
    # across the periodic x face the image at x = 6.5 (distance 0.7) adds in;
    # images further away contribute < 1e-7
    a = (5.8, 0.5, 3.0)
    assert abs(gw(a, (True, True, False)) - gw(a, (False, True, False)) + 2.0 * np.exp(-0.49 / 2.0)) < 1e-7
    # along the Dirichlet z axis no image: making z periodic adds the one at
    # z = 9 (distance 3.2 from z = 5.8)
    b = (0.5, 0.5, 5.8)
    assert abs(gw(b, (True, True, True)) - gw(b, (True, True, False)) + 2.0 * np.exp(-3.2 ** 2 / 2.0)) < 1e-7
