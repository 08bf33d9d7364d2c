"""Pins of the oracle's ChFSI steps: exact filter, QR, brute-force spectra."""
import numpy as np
import pytest

from oracle import chfsi, hamiltonian as ham


@pytest.fixture(scope="module")
def tiny():
    """3^3 cells, p = 3, periodic (729 unknowns), four Gaussian wells."""
    rng = np.random.default_rng(7)
    prob = ham.wells_problem(3, 3, 9.0, True, rng.uniform(0, 9, (4, 3)),
                             rng.uniform(1, 3, 4), rng.uniform(0.8, 1.2, 4))
    H = prob.dense_Htilde()
    evals, evecs = np.linalg.eigh(H)
    return prob, H, evals, evecs


def _cheb(m, x):
    """T_m(x) in closed form: cos(m arccos x) inside [-1, 1], cosh outside."""
    x = np.asarray(x, dtype=float)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1
    out[inside] = np.cos(m * np.arccos(x[inside]))
    ax = np.abs(x[~inside])
    out[~inside] = np.sign(x[~inside]) ** m * np.cosh(m * np.arccosh(ax))
    return out


def test_filter_matches_exact_spectral_filter(tiny):
    prob, H, evals, evecs = tiny
    X = np.random.default_rng(1).uniform(-1, 1, (prob.ndofs, 6))
    a, b, a0 = evals[20], evals[-1] * 1.01, evals[0]
    for m in (1, 2, 7, 25):
        Y = chfsi.chebyshev_filter(prob.apply_Htilde, X, m, a, b, a0)
        Z = chfsi.exact_filter(evals, evecs, X, m, a, b, a0)
        assert np.linalg.norm(Y - Z) <= 1e-10 * np.linalg.norm(Z)


def test_filter_on_eigenvector_is_closed_form_scalar(tiny):
    prob, H, evals, evecs = tiny
    a, b, a0 = evals[15], evals[-1] * 1.02, evals[0]
    c, e = (a + b) / 2, (b - a) / 2
    m = 12
    for i in (0, 5, 40, 300):
        v = evecs[:, i]
        Y = chfsi.chebyshev_filter(prob.apply_Htilde, v[:, None], m, a, b, a0)[:, 0]
        ratio = _cheb(m, (evals[i] - c) / e) / _cheb(m, (a0 - c) / e)
        assert np.linalg.norm(Y - ratio * v) < 1e-11 * max(1.0, abs(ratio))


def test_filter_scalars_reproduce_recurrence(tiny):
    prob, H, evals, evecs = tiny
    X = np.random.default_rng(2).uniform(-1, 1, (prob.ndofs, 3))
    a, b, a0 = evals[10], evals[-1] * 1.05, evals[0]
    c, steps = chfsi.filter_scalars(9, a, b, a0)
    Yp, Y = None, X
    for al, be in steps:
        Yn = al * (H @ Y - c * Y) + (be * Yp if Yp is not None else 0.0)
        Yp, Y = Y, Yn
    Z = chfsi.exact_filter(evals, evecs, X, 9, a, b, a0)
    assert np.linalg.norm(Y - Z) <= 1e-10 * np.linalg.norm(Z)


def test_cholgs_is_thin_qr_with_positive_diagonal():
    X = np.random.default_rng(3).uniform(-1, 1, (500, 40))
    Q = chfsi.cholgs(X)
    assert np.abs(Q.T @ Q - np.eye(40)).max() < 1e-13
    Qr, R = np.linalg.qr(X)
    Qr = Qr * np.sign(np.diag(R))[None, :]
    assert np.abs(Q - Qr).max() < 1e-12


def test_rayleigh_ritz_on_exact_eigenvectors(tiny):
    prob, H, evals, evecs = tiny
    V = evecs[:, :10]
    R = np.linalg.qr(np.random.default_rng(4).standard_normal((10, 10)))[0]
    D, X = chfsi.rayleigh_ritz(prob.apply_Htilde, V @ R)
    assert np.abs(D - evals[:10]).max() < 1e-12
    assert np.abs(np.abs(np.sum(X * V, 0)) - 1).max() < 1e-8


def test_chfsi_converges_to_dense_spectrum_with_interlacing(tiny):
    prob, H, evals, evecs = tiny
    n = 12
    X0 = np.random.default_rng(5).uniform(-1, 1, (prob.ndofs, n + 4))
    b = chfsi.lanczos_upper_bound(prob.apply_Htilde, np.random.default_rng(6).uniform(-1, 1, prob.ndofs), 20)
    assert b >= evals[-1]
    D, X, hist = chfsi.chfsi(prob.apply_Htilde, X0, 15, 25, b, history=True)
    for d in hist:                        # Cauchy interlacing: Ritz values bound from above
        assert np.all(d - evals[:len(d)] > -1e-11)
    assert np.abs(D[:n] - evals[:n]).max() < 1e-10
    r = chfsi.residual_norms(prob.apply_Htilde, X, D)[:n]
    assert r.max() < 1e-6


def test_lanczos_bound_is_an_upper_bound(tiny):
    prob, H, evals, evecs = tiny
    for seed in range(3):
        v0 = np.random.default_rng(seed).uniform(-1, 1, prob.ndofs)
        b = chfsi.lanczos_upper_bound(prob.apply_Htilde, v0, 15)
        assert evals[-1] <= b <= 1.5 * evals[-1]


def test_generalized_residual_equals_direct_definition(tiny):
    prob, H, evals, evecs = tiny
    X = evecs[:, :5] + 1e-4 * np.random.default_rng(8).standard_normal((prob.ndofs, 5))
    lam = evals[:5]
    g = chfsi.generalized_residual_norms(prob.apply_Htilde, X, lam, prob.mass)
    # direct: Psi = M^{-1/2} x / |x|, r = H Psi - lambda M Psi with the assembled H
    Hfull = prob.dense_H()
    Xn = X / np.linalg.norm(X, axis=0)
    Psi = Xn / np.sqrt(prob.mass)[:, None]
    Rd = Hfull @ Psi - prob.mass[:, None] * Psi * lam[None, :]
    assert np.allclose(g, np.linalg.norm(Rd, axis=0), rtol=1e-10, atol=1e-14)
