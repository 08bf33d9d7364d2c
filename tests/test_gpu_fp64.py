"""Parity of the binary64 CUDA path with the FP64 oracle (element by element).

Cases span several cell colours and column tiles with ragged tails: periodic
even and odd cell counts, Dirichlet meshes, projectors, 1..37 columns.
Tolerances: 1e-13 relative Frobenius for one operator application, 1e-12 for
the filtered block (the accuracy the method statement asks of the binary64
path), 1e-10 Ha for eigenvalues.
"""
import numpy as np
import pytest
import torch

from paper_1903_10959_gb300 import ChfsiError, workloads as W
from oracle import chfsi as och

from gpu_util import gpu_context, oracle_problem, rel_fro

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _sys(kind):
    if kind == "c1":
        return W.small_periodic()
    if kind == "odd":          # 3 cells per side periodic: 27 colours
        return W.small_periodic(seed=12, ncell=3, p=3, L=7.5, n_wells=4, n_want=12)
    if kind == "dirichlet":
        s = W.small_periodic(seed=13, ncell=3, p=4, L=9.0, n_wells=5, n_want=12)
        s.periodic = False
        return s
    if kind == "nonlocal":
        s = W.small_periodic(seed=14, ncell=4, p=3, L=10.0, n_wells=6, n_want=16)
        s.nl_centres = s.centres[:3].copy()
        s.nl_h = 0.5 + np.arange(12).reshape(3, 4) / 8.0
        s.nl_rcut = 3.0
        return s
    raise ValueError(kind)


@pytest.fixture(scope="module", params=["c1", "odd", "dirichlet", "nonlocal"])
def case(request):
    s = _sys(request.param)
    prob = oracle_problem(s)
    ctx = gpu_context(s)
    yield s, prob, ctx
    ctx.destroy()


def test_start_block_generator_is_bit_exact():
    s = _sys("c1")
    ctx = gpu_context(s)
    X = torch.empty((ctx.ndofs, 37), dtype=torch.float64, device=DEV)
    ctx.fill_uniform(X, seed=5)
    ref = W.start_block(5, ctx.ndofs, 37)
    assert np.array_equal(X.cpu().numpy(), ref)
    X32 = torch.empty((ctx.ndofs, 37), dtype=torch.float32, device=DEV)
    ctx.fill_uniform(X32, seed=5, prec="mixed")
    assert np.array_equal(X32.cpu().numpy(), ref.astype(np.float32))
    ctx.destroy()


def test_mass_matches_oracle(case):
    s, prob, ctx = case
    assert np.abs(ctx.mass_diag() - prob.mass).max() < 1e-14 * prob.mass.max()


@pytest.mark.parametrize("ncol", [1, 5, 17, 37])
def test_apply_parity(case, ncol):
    s, prob, ctx = case
    X0 = W.start_block(3, prob.ndofs, ncol)
    X = torch.tensor(X0, device=DEV)
    Y = torch.empty_like(X)
    ctx.set_blocking(16, 32)
    ctx.apply(X, Y)
    assert rel_fro(Y.cpu().numpy(), prob.apply_Htilde(X0)) < 1e-13


@pytest.mark.parametrize("degree,block", [(1, 16), (2, 7), (9, 40), (20, 16)])
def test_filter_parity(case, degree, block):
    s, prob, ctx = case
    n = 19
    X0 = W.start_block(4, prob.ndofs, n)
    # fixed bounds from the spectrum scale of the mesh (same numbers on both sides)
    b = och.lanczos_upper_bound(prob.apply_Htilde, W.lanczos_start(4, prob.ndofs), 15)
    a, a0 = 0.2 * b, -3.0
    ref = och.chebyshev_filter(prob.apply_Htilde, X0, degree, a, b, a0)
    X = torch.tensor(X0, device=DEV)
    ctx.set_blocking(block, 32)
    ctx.filter(X, degree, a, b, a0)
    assert rel_fro(X.cpu().numpy(), ref) < 1e-12


def test_filter_strided_columns(case):
    """Filtering a column window of a wider buffer leaves the other columns alone."""
    s, prob, ctx = case
    X0 = W.start_block(6, prob.ndofs, 24)
    b = och.lanczos_upper_bound(prob.apply_Htilde, W.lanczos_start(6, prob.ndofs), 15)
    X = torch.tensor(X0, device=DEV)
    ctx.set_blocking(8, 32)
    ctx.filter(X[:, 5:18], 7, 0.3 * b, b, -2.0)
    out = X.cpu().numpy()
    assert np.array_equal(out[:, :5], X0[:, :5]) and np.array_equal(out[:, 18:], X0[:, 18:])
    ref = och.chebyshev_filter(prob.apply_Htilde, X0[:, 5:18], 7, 0.3 * b, b, -2.0)
    assert rel_fro(out[:, 5:18], ref) < 1e-12


def test_cholgs_parity(case):
    s, prob, ctx = case
    X0 = W.start_block(7, prob.ndofs, 23)
    X = torch.tensor(X0, device=DEV)
    ctx.cholgs(X)
    Q = X.cpu().numpy()
    assert rel_fro(Q, och.cholgs(X0)) < 1e-12
    assert np.abs(Q.T @ Q - np.eye(23)).max() < 1e-13


@pytest.mark.parametrize("n", [1, 31, 32, 33, 65, 200])
def test_cholgs_widths_around_the_inverse_blocks(n):
    """CholGS at widths on both sides of the 32-row blocks of the library's
    triangular inverse (one column, one short block, exactly one block, one
    block and a row, several blocks with a ragged tail) against the oracle's
    CholGS (Algorithm CholGS), and the block's orthonormality."""
    s = _sys("c1")
    ctx = gpu_context(s)
    try:
        X0 = W.start_block(40 + n, ctx.ndofs, n)
        X = torch.tensor(X0, device=DEV)
        ctx.cholgs(X)
        Q = X.cpu().numpy()
        assert rel_fro(Q, och.cholgs(X0)) < 1e-12
        assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-13
    finally:
        ctx.destroy()


def test_rayleigh_ritz_parity(case):
    s, prob, ctx = case
    X0 = och.cholgs(W.start_block(8, prob.ndofs, 21))
    D_ref, Xr = och.rayleigh_ritz(prob.apply_Htilde, X0)
    X = torch.tensor(X0, device=DEV)
    ctx.set_blocking(8, 32)
    D = ctx.rayleigh_ritz(X)
    assert np.abs(D - D_ref).max() < 1e-10
    Xg = X.cpu().numpy()
    # columns agree up to sign where the Ritz values are isolated
    gaps = np.minimum(np.diff(D_ref, prepend=-np.inf), np.diff(D_ref, append=np.inf))
    iso = gaps > 1e-6
    ov = np.abs(np.sum(Xg * Xr, axis=0))
    assert np.abs(ov[iso] - 1).max() < 1e-9


def test_solve_eigenvalues_match_oracle(case):
    s, prob, ctx = case
    n = s.n_sub
    iters = 4
    X0 = W.start_block(s.seed, prob.ndofs, n)
    b = och.lanczos_upper_bound(prob.apply_Htilde, W.lanczos_start(s.seed, prob.ndofs), 20)
    D_ref, X_ref = och.chfsi(prob.apply_Htilde, X0, s.degree, iters, b)
    X = torch.tensor(X0, device=DEV)
    ctx.set_blocking(200, 32)
    D, done = ctx.solve(X, iters, s.degree, b)
    assert done == iters
    assert np.abs(D - D_ref).max() < 1e-10
    r, g = ctx.residuals(X, D)
    r_ref = och.residual_norms(prob.apply_Htilde, X_ref, D_ref)
    assert np.allclose(r, r_ref, rtol=1e-6, atol=1e-12)


def test_bounds_match_oracle_lanczos(case):
    s, prob, ctx = case
    b = ctx.bounds(steps=20, seed=9)
    ref = och.lanczos_upper_bound(prob.apply_Htilde, W.lanczos_start(9, prob.ndofs), 20)
    assert abs(b - ref) < 1e-9 * abs(ref)


def test_cholgs_rank_deficient_reports_not_spd():
    s = _sys("c1")
    ctx = gpu_context(s)
    X0 = W.start_block(2, ctx.ndofs, 6)
    X0[:, 3] = X0[:, 1]
    X = torch.tensor(X0, device=DEV)
    with pytest.raises(ChfsiError) as ei:
        ctx.cholgs(X)
    assert ei.value.status == 4
    assert np.array_equal(X.cpu().numpy(), X0)       # X left unchanged
    ctx.destroy()
