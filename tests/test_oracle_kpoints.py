"""Pins of the Bloch-periodic oracle H~(k) (Eq. evp of Eq. ksproblemPer):
k = 0 reduces to the real Hamiltonian, the assembled operator is Hermitian,
time reversal maps k to -k, the free particle gives 1/2 |2 pi n / L + k|^2,
and the bands are periodic in k up to the FE error."""
import numpy as np
import pytest

from oracle import hamiltonian as oh
from oracle import kpoints as kp


def _wells(L=6.0, n=3, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, L, (n, 3)), rng.uniform(1, 3, n), rng.uniform(0.8, 1.2, n)


def test_k_zero_is_the_real_hamiltonian():
    c, d, w = _wells()
    prob = oh.wells_problem(2, 3, 6.0, True, c, d, w)
    X = np.random.default_rng(1).uniform(-1, 1, (prob.ndofs, 4))
    got = kp.BlochProblem(prob, [0.0, 0.0, 0.0]).apply_Htilde(X)
    assert np.abs(got.imag).max() == 0.0
    assert np.allclose(got.real, prob.apply_Htilde(X), rtol=0, atol=1e-13)


def test_hermitian_and_time_reversal():
    c, d, w = _wells()
    prob = oh.wells_problem(2, 3, 6.0, True, c, d, w)
    k = np.array([0.31, -0.17, 0.44])
    H = kp.BlochProblem(prob, k).dense_Htilde()
    scale = np.abs(H).max()
    assert np.abs(H - H.conj().T).max() < 1e-13 * scale      # -i k.G is Hermitian once assembled
    assert np.abs(H.imag).max() > 1e-3 * scale                 # and not trivially real
    Hm = kp.BlochProblem(prob, -k).dense_Htilde()
    assert np.abs(Hm - H.conj()).max() < 1e-14 * scale
    ev = np.linalg.eigvalsh(H)
    assert np.allclose(np.linalg.eigvalsh(Hm), ev, rtol=0, atol=1e-11)


def _free_levels(L, k, nmax=3):
    g = 2 * np.pi / L
    n = np.arange(-nmax, nmax + 1)
    G = np.stack(np.meshgrid(n, n, n, indexing="ij"), -1).reshape(-1, 3) * g
    return np.sort(0.5 * np.sum((G + k) ** 2, axis=1))


@pytest.mark.parametrize("k", [[0.2, 0.0, 0.0], [0.25, -0.4, 0.1]])
def test_free_particle_bands(k):
    L = 6.0
    prob = oh.Problem(3, 4, L, True, lambda x: np.zeros(len(x)))
    k = np.asarray(k)
    ev = np.linalg.eigvalsh(kp.BlochProblem(prob, k).dense_Htilde())
    ref = _free_levels(L, k)
    assert np.allclose(ev[:12], ref[:12], rtol=2e-3)


def test_shift_by_a_reciprocal_vector_preserves_the_low_bands():
    """eps(k + G) = eps(k) in the continuum; in the FE space the gauge factor
    exp(i G.x) is only approximated, so the low bands agree to FE accuracy,
    which improves with the degree (same number of unknowns: 3 cells at p = 4,
    2 cells at p = 6)."""
    L = 6.0
    k = np.array([0.2, 0.1, 0.0])
    gap = []
    for ncell, p in ((3, 4), (2, 6)):
        prob = oh.Problem(ncell, p, L, True, lambda x: np.zeros(len(x)))
        e1 = np.linalg.eigvalsh(kp.BlochProblem(prob, k).dense_Htilde())[:6]
        e2 = np.linalg.eigvalsh(kp.BlochProblem(prob, k + [2 * np.pi / L, 0, 0]).dense_Htilde())[:6]
        gap.append(np.abs(e1 - e2).max() / np.abs(e1).max())
    assert gap[0] < 1e-2 and gap[1] < 2e-3 and gap[1] < gap[0] / 4
