"""The BF16x3 cell kernel variants -- the bulk-async-copy gather, the
decoupled matrix / Y rings, the whole cell per CTA and several column tiles
per CTA -- give the same bits as the register gather
(same split, same MMA order, same tiling), for every
FE degree the kernel plans for, Dirichlet rows, ragged last column tiles and
several 128-column tiles; an unaligned block falls back to the register
gather.  Both are checked against the oracle's H~ X as well."""
import numpy as np
import pytest
import torch

from paper_1903_10959_gb300 import workloads as W

from gpu_util import gpu_context, oracle_problem, rel_fro

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _sys(p, periodic=True):
    s = W.small_periodic(seed=130 + p, ncell=3 if p <= 5 else 2, p=p, L=6.0, n_wells=4, n_want=10)
    if not periodic:
        s.periodic = False
        s.centres = 0.1 * s.L + 0.8 * s.centres
    return s


def _apply(ctx, X, mode):
    ctx.set_cell_gather(mode)
    Y = torch.empty_like(X)
    ctx.apply(X, Y, prec="bf16x3")
    return Y


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("periodic", [True, False])
def test_async_gather_is_bit_identical(p, periodic):
    s = _sys(p, periodic)
    ctx = gpu_context(s)
    prob = oracle_problem(s)
    try:
        for ncol in (4, 132, 260, 520):            # one ragged tile, 2, 3 and 5 tiles
            x = W.start_block(ncol, ctx.ndofs, ncol).astype(np.float32)
            X = torch.tensor(x, device=DEV)
            ya = _apply(ctx, X, "async")
            yr = _apply(ctx, X, "registers")
            yg = _apply(ctx, X, "rings")
            y4 = _apply(ctx, X, "rings4")
            yw = _apply(ctx, X, "whole")
            yt = _apply(ctx, X, "tiles")              # 3 tiles per CTA: groups of 1, 2, 3, 3 + 2
            y2 = _apply(ctx, X, "tiles2")             # all tiles per CTA, two accumulators
            assert torch.equal(yw, yr), (p, periodic, ncol)
            assert torch.equal(y2, yr), (p, periodic, ncol)
            assert torch.equal(yt, yr), (p, periodic, ncol)
            assert torch.equal(ya, yr), (p, periodic, ncol)
            assert torch.equal(yg, yr), (p, periodic, ncol)
            assert torch.equal(y4, yr), (p, periodic, ncol)
            if ncol == 4:
                ref = prob.apply_Htilde(x.astype(np.float64))
                assert rel_fro(ya.cpu().numpy().astype(np.float64), ref) < 1e-5
    finally:
        ctx.destroy()


def test_unaligned_block_falls_back():
    s = _sys(4)
    ctx = gpu_context(s)
    try:
        x = W.start_block(3, ctx.ndofs, 7).astype(np.float32)
        X = torch.tensor(x, device=DEV)                   # 7 columns: rows not 16-byte multiples
        assert torch.equal(_apply(ctx, X, "async"), _apply(ctx, X, "registers"))
        wide = torch.zeros((ctx.ndofs, 9), device=DEV)
        wide[:, :8] = torch.tensor(W.start_block(4, ctx.ndofs, 8).astype(np.float32), device=DEV)
        V = wide[:, :8]                                   # ldx = 9: rows not 16-byte aligned
        assert torch.equal(_apply(ctx, V, "async"), _apply(ctx, V, "registers"))
    finally:
        ctx.destroy()


@pytest.mark.parametrize("p", [3, 5, 7])
def test_projector_chunks_in_the_ring_kernel(p):
    """With projectors, the ring kernels add the expansion C~ h Z as extra
    K-chunks of each cell's product (the owned rows' share) instead of in the
    assembly: against the oracle's H~ X (1e-5, as every BF16x3 apply) and the
    register-gather path, whose assembly adds the same term (1e-6)."""
    s = W.small_periodic(seed=170 + p, ncell=3 if p <= 5 else 2, p=p, L=7.0, n_wells=4, n_want=10)
    s.nl_centres = s.centres[:3].copy()
    s.nl_h = 0.5 + np.arange(12).reshape(3, 4) / 8.0
    s.nl_rcut = 2.5
    ctx = gpu_context(s)
    prob = oracle_problem(s)
    try:
        for ncol in (4, 132):
            x = W.start_block(ncol + 1, ctx.ndofs, ncol).astype(np.float32)
            X = torch.tensor(x, device=DEV)
            yg = _apply(ctx, X, "rings")
            y4 = _apply(ctx, X, "rings4")
            yr = _apply(ctx, X, "registers")
            assert torch.equal(yg, y4)
            ref = prob.apply_Htilde(x.astype(np.float64))
            assert rel_fro(yg.cpu().numpy().astype(np.float64), ref) < 1e-5
            assert rel_fro(yg.cpu().numpy().astype(np.float64), yr.cpu().numpy().astype(np.float64)) < 1e-6
    finally:
        ctx.set_cell_gather("rings")
        ctx.destroy()
