"""chfsi_apply_noalloc: H~ X without device allocation, against the oracle's
H~ X (Eqs. discreteHam, nonlocalHamDiscrete in the standard form of Eq. hep)
and against chfsi_apply.

The no-allocation entry point is for callers that cannot call cudaMalloc
inside their step (a host framework whose own pool allocator owns the GPU's
memory, or a latency-critical loop where cudaMalloc / cudaFree would
synchronise the device).  Its assembly scratch is the library's fixed 64 MiB
device array.  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes alone in a
fresh process.  Tolerance: the 1e-13 relative Frobenius bound the binary64
apply tests use.
"""
import numpy as np
import pytest
import torch

from paper_1903_10959_gb300 import ChfsiError, workloads as W

from gpu_util import gpu_context, oracle_problem, rel_fro

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _systems():
    s = W.small_periodic(seed=31, ncell=4, p=4, L=10.0, n_wells=6, n_want=12)
    t = W.small_periodic(seed=32, ncell=3, p=3, L=9.0, n_wells=4, n_want=12)
    t.nl_centres = t.centres[:2].copy()
    t.nl_h = 0.5 + np.arange(8).reshape(2, 4) / 8.0
    return [s, t]


@pytest.mark.parametrize("which", [0, 1])
def test_noalloc_apply_matches_apply_twice(which):
    s = _systems()[which]
    ctx = gpu_context(s)
    try:
        ncol = 37
        X0 = W.start_block(5, ctx.ndofs, ncol)
        X = torch.tensor(X0, device=DEV)
        Yref = torch.empty_like(X)
        ctx.apply(X, Yref)
        ref = Yref.cpu().numpy()
        oracle = oracle_problem(s).apply_Htilde(X0)
        for _ in range(2):            # the shared scratch keeps the last call's contents
            Y = torch.full_like(X, float("nan"))
            ctx.apply_noalloc(X, Y)
            got = Y.cpu().numpy()
            assert rel_fro(got, oracle) <= 1e-13
            assert rel_fro(got, ref) <= 1e-13
    finally:
        ctx.destroy()


def test_noalloc_rejects_oversize_request():
    s = _systems()[0]
    ctx = gpu_context(s)
    try:
        ncol = (64 << 20) // (8 * ctx.ndofs) + 1     # one column more than the 64 MiB scratch holds
        X = torch.zeros((ctx.ndofs, ncol), dtype=torch.float64, device=DEV)
        Y = torch.zeros_like(X)
        with pytest.raises(ChfsiError) as ei:
            ctx.apply_noalloc(X, Y)
        assert ei.value.status == 1 and "bytes of scratch" in str(ei.value)
    finally:
        ctx.destroy()
