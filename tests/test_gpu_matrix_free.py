"""Parity of the matrix-free (sum-factorised) binary64 cell apply with the
FP64 oracle: the oracle's own matrix-free apply (oracle/matrix_free.py) and
its dense assembled apply, element by element.

Cases span FE degrees 2..8 (every instantiated kernel), periodic, Dirichlet
and semi-periodic meshes, several colours and ragged column tiles, and the
projector term.  Tolerances as for the binary64 path: 1e-13 relative for one
application, 1e-12 for the filtered block, 1e-10 Ha for eigenvalues.
"""
import numpy as np
import pytest
import torch

from paper_1903_10959_gb300 import ChfsiError, workloads as W
from oracle import chfsi as och
from oracle import matrix_free as omf

from gpu_util import gpu_context, oracle_problem, rel_fro

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _sys(kind, p=3):
    if kind == "periodic":
        return W.small_periodic(seed=90 + p, ncell=3 if p <= 5 else 2, p=p, L=6.0, n_wells=4, n_want=10)
    if kind == "dirichlet":
        s = W.small_periodic(seed=100 + p, ncell=3, p=p, L=7.0, n_wells=3, n_want=10)
        s.periodic = False
        s.centres = 0.1 * s.L + 0.8 * s.centres
        return s
    if kind == "slab":
        s = W.small_periodic(seed=110 + p, ncell=3, p=p, L=6.0, n_wells=3, n_want=10)
        s.periodic = (True, False, True)
        return s
    if kind == "nonlocal":
        s = W.small_periodic(seed=120 + p, ncell=4, p=p, L=10.0, n_wells=6, n_want=16)
        s.nl_centres = s.centres[:3].copy()
        s.nl_h = 0.5 + np.arange(12).reshape(3, 4) / 8.0
        s.nl_rcut = 3.0
        return s
    raise ValueError(kind)


def _ctx_mf(s):
    ctx = gpu_context(s)
    ctx.set_fp64_operator("matrix-free")
    assert ctx.fp64_operator == "matrix-free"
    return ctx


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7, 8])
def test_apply_matches_oracle_every_degree(p):
    s = _sys("periodic", p)
    prob = oracle_problem(s)
    ctx = _ctx_mf(s)
    try:
        for ncol in (1, 3, 9):
            X0 = W.start_block(3 + ncol, prob.ndofs, ncol)
            Y = torch.empty((prob.ndofs, ncol), dtype=torch.float64, device=DEV)
            ctx.apply(torch.tensor(X0, device=DEV), Y)
            got = Y.cpu().numpy()
            ref = prob.apply_Htilde(X0)
            assert rel_fro(got, ref) < 1e-13
            assert np.abs(got - omf.apply_Htilde(prob, X0)).max() < 1e-13 * np.abs(ref).max()
    finally:
        ctx.destroy()


@pytest.fixture(scope="module", params=["periodic", "dirichlet", "slab", "nonlocal"])
def case(request):
    s = _sys(request.param, 4)
    prob = oracle_problem(s)
    ctx = _ctx_mf(s)
    yield s, prob, ctx
    ctx.destroy()


@pytest.mark.parametrize("ncol", [1, 5, 17, 37])
def test_apply_parity(case, ncol):
    s, prob, ctx = case
    X0 = W.start_block(4, prob.ndofs, ncol)
    X = torch.tensor(X0, device=DEV)
    Y = torch.empty_like(X)
    ctx.set_blocking(16, 32)
    ctx.apply(X, Y)
    assert rel_fro(Y.cpu().numpy(), prob.apply_Htilde(X0)) < 1e-13


def test_matches_cell_matrix_operator(case):
    s, prob, ctx = case
    X0 = W.start_block(6, prob.ndofs, 11)
    X = torch.tensor(X0, device=DEV)
    Ymf, Ycm = torch.empty_like(X), torch.empty_like(X)
    ctx.apply(X, Ymf)
    ctx.set_fp64_operator("cells")
    ctx.apply(X, Ycm)
    ctx.set_fp64_operator("matrix-free")
    assert rel_fro(Ymf.cpu().numpy(), Ycm.cpu().numpy()) < 1e-13


@pytest.mark.parametrize("degree,block", [(2, 7), (10, 16)])
def test_filter_parity(case, degree, block):
    s, prob, ctx = case
    X0 = W.start_block(5, prob.ndofs, 23)
    ctx.set_blocking(block, 32)
    X = torch.tensor(X0, device=DEV)
    a, b, a0 = 4.0, 80.0, -3.0
    ctx.filter(X, degree, a, b, a0)
    ref = och.chebyshev_filter(prob.apply_Htilde, X0, degree, a, b, a0)
    assert rel_fro(X.cpu().numpy(), ref) < 1e-12


def test_solve_eigenvalues(case):
    s, prob, ctx = case
    b = och.lanczos_upper_bound(prob.apply_Htilde, W.lanczos_start(s.seed, prob.ndofs), 20)
    X0 = W.start_block(s.seed, prob.ndofs, s.n_sub)
    D_ref, _ = och.chfsi(prob.apply_Htilde, X0, 12, 4, b)
    ctx.set_blocking(200, 32)
    X = torch.tensor(X0, device=DEV)
    D, _ = ctx.solve(X, 4, 12, b)
    assert np.abs(D - D_ref).max() < 1e-10


def test_unsupported_rule_is_rejected():
    s = _sys("periodic", 3)
    from paper_1903_10959_gb300 import Context
    ctx = Context(s.ncell, s.L, s.p, periodic=True, quad_points=s.p + 3)
    try:
        with pytest.raises(ChfsiError):
            ctx.set_fp64_operator("matrix-free")
        assert ctx.fp64_operator == "cells"
    finally:
        ctx.destroy()
