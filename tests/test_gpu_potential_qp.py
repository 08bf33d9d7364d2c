"""General effective potential at the Gauss points (chfsi_set_potential_qp)
against the oracle built with the same V_eff as a callable (Eq. discreteHam:
V_e = int V N_j N_k by the Gauss rule of the cell)."""
import numpy as np
import pytest
import torch

from oracle import hamiltonian as oham
from paper_1903_10959_gb300 import ChfsiError, Context, workloads as W

from gpu_util import rel_fro

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _points(prob):
    """(ncells * q^3, 3) Gauss points, cells x fastest, point a + q (b + q c)."""
    return np.concatenate([prob.basis.quad_coords(prob.mesh.cell_origin(e))
                           for e in range(prob.mesh.ncells)])


def _field(L):
    k = 2.0 * np.pi / L
    return lambda x: 0.4 * np.cos(k * x[:, 0]) + 0.25 * np.sin(k * (x[:, 1] + 2.0 * x[:, 2])) - 0.1


@pytest.fixture(scope="module")
def case():
    s = W.small_periodic(seed=41, ncell=3, p=5, L=7.5, n_wells=3, n_want=8)
    f = _field(s.L)
    wells = lambda x: oham.gaussian_wells(x, s.centres, s.depths, s.widths, s.L, True)
    prob = oham.Problem(s.ncell, s.p, s.L, True, lambda x: wells(x) + f(x))
    return s, prob, f, wells


def _ctx(s, wells=True, vqp=None):
    ctx = Context(s.ncell, s.L, s.p, periodic=True)
    if wells:
        ctx.set_potential_gaussians(s.centres, s.depths, s.widths)
    if vqp is not None:
        ctx.set_potential_qp(vqp)
    ctx.build()
    return ctx


def test_field_plus_wells_matches_oracle(case):
    s, prob, f, _ = case
    X0 = W.start_block(7, prob.ndofs, 37)
    ref = prob.apply_Htilde(X0)
    with _ctx(s, vqp=f(_points(prob))) as ctx:
        X = torch.tensor(X0, device=DEV)
        Y = torch.empty_like(X)
        ctx.apply(X, Y)
        assert rel_fro(Y.cpu().numpy(), ref) < 1e-12
        # the BF16x3 tensor-core path on the same cell matrices
        X32 = torch.tensor(X0.astype(np.float32), device=DEV)
        Y32 = torch.empty_like(X32)
        ctx.apply(X32, Y32, prec="bf16x3")
        ref32 = prob.apply_Htilde(X0.astype(np.float32).astype(np.float64))
        assert rel_fro(Y32.cpu().numpy().astype(np.float64), ref32) < 1e-5


def test_wells_as_values_equal_wells(case):
    """The wells given as Gauss-point values instead of centres: the same cell
    matrices up to the rounding of the exponentials."""
    s, prob, _, wells = case
    X0 = W.start_block(8, prob.ndofs, 20)
    X = torch.tensor(X0, device=DEV)
    Ya, Yb = torch.empty_like(X), torch.empty_like(X)
    with _ctx(s) as ca:
        ca.apply(X, Ya)
    with _ctx(s, wells=False, vqp=wells(_points(prob))) as cb:
        cb.apply(X, Yb)
    assert rel_fro(Yb.cpu().numpy(), Ya.cpu().numpy()) < 1e-13


def test_clear_and_bad_count(case):
    s, prob, f, _ = case
    X0 = W.start_block(9, prob.ndofs, 5)
    X = torch.tensor(X0, device=DEV)
    Ya, Yb = torch.empty_like(X), torch.empty_like(X)
    with _ctx(s) as ca:
        ca.apply(X, Ya)
    with _ctx(s, vqp=f(_points(prob))) as cb:
        cb.set_potential_qp(None)            # cleared: the wells alone again
        cb.build()
        cb.apply(X, Yb)
        assert rel_fro(Yb.cpu().numpy(), Ya.cpu().numpy()) < 1e-15
        with pytest.raises(ChfsiError):
            cb.set_potential_qp(np.zeros(7))
