"""Semi-periodic systems (per-axis boundary conditions, Sec. 1): a slab,
periodic in x and y with Dirichlet faces normal to z, and a wire, periodic in
y only, with wells and projectors, against the oracle."""
import numpy as np
import pytest
import torch

from oracle import chfsi as och
from oracle import hamiltonian as oham
from paper_1903_10959_gb300 import Context, workloads as W

from gpu_util import rel_fro

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", params=[(True, True, False), (False, True, False)], ids=["slab", "wire"])
def case(request):
    per = request.param
    s = W.small_periodic(seed=51, ncell=3, p=4, L=7.5, n_wells=4, n_want=10, degree=12)
    nl_c = s.centres[:2].copy()
    nl_h = 0.5 + np.arange(8).reshape(2, 4) / 6.0
    proj = dict(centres=nl_c, sigma=0.8, rcut=3.0, h=nl_h)
    prob = oham.wells_problem(s.ncell, s.p, s.L, per, s.centres, s.depths, s.widths, projectors=proj)
    ctx = Context(s.ncell, s.L, s.p, periodic=per)
    ctx.set_potential_gaussians(s.centres, s.depths, s.widths)
    ctx.set_projectors(nl_c, nl_h, 0.8, 3.0)
    ctx.build()
    yield s, prob, ctx
    ctx.destroy()


def test_unknowns_and_mass(case):
    s, prob, ctx = case
    assert ctx.ndofs == prob.ndofs
    assert np.abs(ctx.mass_diag() - prob.mass).max() < 1e-14 * prob.mass.max()


@pytest.mark.parametrize("ncol", [1, 19])
def test_apply_parity(case, ncol):
    s, prob, ctx = case
    X0 = W.start_block(3, prob.ndofs, ncol)
    X = torch.tensor(X0, device=DEV)
    Y = torch.empty_like(X)
    ctx.apply(X, Y)
    assert rel_fro(Y.cpu().numpy(), prob.apply_Htilde(X0)) < 1e-12
    X32 = torch.tensor(X0.astype(np.float32), device=DEV)
    Y32 = torch.empty_like(X32)
    ctx.apply(X32, Y32, prec="bf16x3")
    ref = prob.apply_Htilde(X0.astype(np.float32).astype(np.float64))
    assert rel_fro(Y32.cpu().numpy().astype(np.float64), ref) < 1e-5


def test_solve_eigenvalues_match_oracle(case):
    s, prob, ctx = case
    n, iters = s.n_sub, 3
    X0 = W.start_block(s.seed, prob.ndofs, n)
    b = och.lanczos_upper_bound(prob.apply_Htilde, W.lanczos_start(s.seed, prob.ndofs), 20)
    D_ref, _ = och.chfsi(prob.apply_Htilde, X0, s.degree, iters, b)
    X = torch.tensor(X0, device=DEV)
    D, done = ctx.solve(X, iters, s.degree, b)
    assert done == iters
    assert np.abs(D - D_ref).max() < 1e-10
