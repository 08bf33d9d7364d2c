"""Bounded device waits: a BF16x3 cell-kernel launch whose gather warp
withholds one barrier arrival (test hook chfsi_debug_withhold_arrival) makes
the MMA warp's wait run out after its 2 s limit.  The kernel unwinds (waits
for its own bulk copies, frees its TMEM), the call returns
CHFSI_ERR_TIMEOUT, and the context stays usable: with the hook off, the next
application gives the oracle's result."""
import numpy as np
import pytest
import torch

from paper_1903_10959_gb300 import ChfsiError, workloads as W

from gpu_util import gpu_context, oracle_problem, rel_fro

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_withheld_arrival_times_out_and_context_recovers():
    s = W.small_periodic(seed=71, ncell=3, p=4, L=7.5, n_wells=3, n_want=24, degree=8, iters=2)
    ctx = gpu_context(s)
    try:
        M, n = ctx.ndofs, s.n_sub
        x = W.start_block(s.seed, M, n).astype(np.float32)
        X = torch.tensor(x, device=DEV)
        Y = torch.empty_like(X)
        ctx.apply(X, Y, prec="bf16x3")                       # packs the cell data first
        ctx.debug_withhold_arrival(True)
        try:
            with pytest.raises(ChfsiError) as ei:
                ctx.apply(X, Y, prec="bf16x3")
        finally:
            ctx.debug_withhold_arrival(False)
        assert ei.value.status == 7                          # CHFSI_ERR_TIMEOUT
        assert "timed out" in str(ei.value)
        # the same context, hook off: correct again
        ctx.apply(X, Y, prec="bf16x3")
        ref = oracle_problem(s).apply_Htilde(x.astype(np.float64))
        assert rel_fro(Y.cpu().numpy().astype(np.float64), ref) < 1e-5
        # and the other paths on it still run
        Z = torch.tensor(x.astype(np.float64), device=DEV)
        ctx.cholgs(Z, prec="fp64")
        q = Z.cpu().numpy()
        assert np.abs(q.T @ q - np.eye(n)).max() < 1e-12
    finally:
        ctx.destroy()
