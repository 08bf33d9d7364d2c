"""The 256-row tile kernel of the mixed-precision rotations X U (CholGS and
Rayleigh-Ritz, Sec. 3.3.2-3.3.3) against the 128 x 128 tile kernel and the
oracle, forced on small systems so that row blocks, column tiles and the
upper-triangular (X L^{-T}) form all have ragged edges: 3,375 unknowns (not a
multiple of 256), block widths 1, 37 (one tile of 48 columns), 300 (two
tiles of 160, the second ragged) and 520 (three tiles of 176).

Tolerances: the two kernels accumulate the same products in the same order
per output element; 1e-6 relative between them, and the mixed CholGS /
Rayleigh-Ritz bars of the other mixed-precision tests against the oracle.
"""
import numpy as np
import pytest
import torch

from paper_1903_10959_gb300 import ChfsiError, workloads as W
from oracle import chfsi as och

from gpu_util import gpu_context, oracle_problem, rel_fro

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def case():
    s = W.small_periodic(seed=33, ncell=5, p=3, L=8.0, n_wells=5, n_want=20)
    prob = oracle_problem(s)
    ctx = gpu_context(s)
    assert ctx.ndofs == 3375
    yield s, prob, ctx
    ctx.set_gemm_kernels(-1, -1)
    ctx.destroy()


@pytest.mark.parametrize("n", [1, 37, 300, 520])
@pytest.mark.parametrize("prec", ["mixed", "bf16x3"])
@pytest.mark.parametrize("bd", [1, 8])
def test_cholgs_wide_matches_narrow_and_oracle(case, n, prec, bd):
    s, prob, ctx = case
    X0 = W.start_block(70 + n, prob.ndofs, n).astype(np.float32)
    ctx.set_blocking(200, bd)
    out = {}
    for k in (0, 1):
        ctx.set_gemm_kernels(tall=k)
        X = torch.tensor(X0, device=DEV)
        ctx.cholgs(X, prec=prec)
        out[k] = X.cpu().numpy().astype(np.float64)
    ctx.set_gemm_kernels(-1, -1)
    assert rel_fro(out[1], out[0]) < 1e-6
    Q = out[1]
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 2e-5
    assert rel_fro(Q, och.cholgs(X0.astype(np.float64))) < 2e-5


@pytest.mark.parametrize("n", [37, 300])
@pytest.mark.parametrize("prec", ["mixed", "bf16x3"])
def test_rayleigh_ritz_wide_matches_narrow_and_oracle(case, n, prec):
    s, prob, ctx = case
    X0 = och.cholgs(W.start_block(80 + n, prob.ndofs, n)).astype(np.float32)
    D_ref, V_ref = och.rayleigh_ritz(prob.apply_Htilde, X0.astype(np.float64))
    ctx.set_blocking(64, 1)
    out, D = {}, {}
    for k in (0, 1):
        ctx.set_gemm_kernels(tall=k)
        X = torch.tensor(X0, device=DEV)
        D[k] = ctx.rayleigh_ritz(X, prec=prec)
        out[k] = X.cpu().numpy().astype(np.float64)
    ctx.set_gemm_kernels(-1, -1)
    assert np.array_equal(D[0], D[1])          # the projected matrix does not use the rotation
    assert rel_fro(out[1], out[0]) < 1e-6
    scale = max(1.0, np.abs(D_ref).max())
    assert np.abs(D[1] - D_ref).max() < 1e-5 * scale


def test_bad_kernel_choice_is_rejected(case):
    s, prob, ctx = case
    with pytest.raises(ChfsiError):
        ctx.set_gemm_kernels(tall=2)
    with pytest.raises(ChfsiError):
        ctx.set_gemm_kernels(gram=-2)
