"""Pins of the SCF oracle (Algorithm scf around the ChFSI step): the periodic
Poisson solve against a single Fourier mode, the exchange potential as the
derivative of its energy density, Anderson mixing's finite termination on a
linear fixed point, and a converged Gaussian-charge system's charge,
self-consistency and mirror symmetry."""
import numpy as np
import pytest

from oracle import scf


def _mode_error(ncell, p, L=6.0, amp=0.7):
    prob = scf.FieldProblem(ncell, p, L, True)
    xq = scf.gauss_points(prob)
    k = 2 * np.pi / L
    f = amp * np.cos(k * xq[..., 0])
    phi = scf.poisson_periodic(prob, f)
    exact = 4 * np.pi * amp / k ** 2 * np.cos(k * prob.mesh.dof_coords()[:, 0])
    return np.abs(phi - exact).max() / np.abs(exact).max(), prob, phi


def test_poisson_single_mode():
    e4, prob, phi = _mode_error(3, 4)
    e6, _, _ = _mode_error(2, 6)
    assert e4 < 1e-3 and e6 < e4 / 3            # FE accuracy, improving with the degree
    m = scf.load_vector(prob, np.ones((prob.mesh.ncells, prob.basis.N.shape[0])))
    assert abs(m @ phi) < 1e-12 * np.abs(phi).max() * m.sum()   # int phi = 0


def test_poisson_neutralises_net_charge():
    prob = scf.FieldProblem(2, 3, 5.0, True)
    nq = prob.basis.N.shape[0]
    f = np.full((prob.mesh.ncells, nq), 0.3)       # a uniform charge is all background
    assert np.abs(scf.poisson_periodic(prob, f)).max() < 1e-12


def test_exchange_potential_is_the_energy_derivative():
    rho = np.array([1e-3, 0.05, 0.4, 2.0])
    h = 1e-6 * rho
    e = lambda r: r * scf.lda_exchange_energy_density(r)
    fd = (e(rho + h) - e(rho - h)) / (2 * h)
    assert np.allclose(scf.lda_exchange_potential(rho), fd, rtol=1e-7)


def test_exchange_energy_of_the_uniform_gas():
    """Dirac exchange of the uniform electron gas: the energy per electron is
    -(3/4)(9 / (4 pi^2))^{1/3} / r_s = -0.4581652932831429 / r_s Ha, with
    rho = 3 / (4 pi r_s^3) (the textbook constant of the local density
    approximation's exchange part)."""
    for rs in (0.5, 1.0, 2.0, 5.0):
        rho = 3.0 / (4.0 * np.pi * rs ** 3)
        assert scf.lda_exchange_energy_density(np.array([rho]))[0] * rs == pytest.approx(-0.4581652932831429,
                                                                                       rel=1e-13)


def test_anderson_terminates_on_a_linear_fixed_point():
    """Anderson mixing with full history on x = G x + c is GMRES on
    (I - G) x = c: exact after at most n + 1 steps."""
    rng = np.random.default_rng(3)
    n = 6
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    G = Q @ np.diag(np.linspace(-0.95, 0.95, n)) @ Q.T
    c = rng.standard_normal(n)
    x_star = np.linalg.solve(np.eye(n) - G, c)
    mix = scf.Anderson(beta=1.0, depth=n + 2)
    x = np.zeros(n)
    for _ in range(n + 2):
        x = mix.step(x, G @ x + c)
    assert np.abs(x - x_star).max() < 1e-10 * np.abs(x_star).max()
    y = np.zeros(n)
    for _ in range(n + 2):                       # plain iteration is far from converged
        y = G @ y + c
    assert np.abs(y - x_star).max() > 1e-2 * np.abs(x_star).max()


@pytest.fixture(scope="module")
def helium():
    return scf.scf(3, 4, 6.0, [[3.0, 3.0, 3.0]], [2.0], [0.6], n_states=4, kT=0.01, degree=20,
                   passes=2, tol=1e-9, max_iter=40)


def test_scf_converges_and_keeps_the_charge(helium):
    r = helium
    assert r["residuals"][-1] < 1e-9 and len(r["residuals"]) < 40
    W = r["problem"].basis.W
    assert abs(np.sum(r["rho"] * W[None, :]) - 2.0) < 1e-3          # GLL lumping error only
    assert abs(r["occ"].sum() - 1.0) < 1e-12                         # 2 sum f = N_e
    assert r["evals"][0] < 0.0                                        # bound by the nucleus


def test_scf_is_self_consistent(helium):
    r = helium
    prob = r["problem"]
    phi = scf.poisson_periodic(prob, r["rho"] + r["bq"])
    vq = scf.nodal_to_gauss(prob, phi) + scf.lda_exchange_potential(r["rho"])
    assert np.abs(vq - r["vq"]).max() < 1e-6 * np.abs(r["vq"]).max()


def test_scf_density_has_the_mirror_symmetry_of_the_system(helium):
    """Nucleus at the centre of a mesh symmetric under x -> L - x: the
    converged density at mirrored Gauss points agrees."""
    r = helium
    prob = r["problem"]
    n, q = prob.mesh.ncell, prob.basis.q
    rho = r["rho"].reshape(n, n, n, q, q, q)          # [cz, cy, cx, c, b, a]
    mirrored = rho[:, :, ::-1, :, :, ::-1]             # x -> L - x
    assert np.abs(mirrored - rho).max() < 1e-6 * np.abs(rho).max()
