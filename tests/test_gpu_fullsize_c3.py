"""Parity of one BF16x3 H~ application on the largest single-GPU workload:
20^3 cells, p = 7 (n_e = 512: the cell rows split into two parts of 256, the
widest MMA the cell kernel issues), 2,744,000 unknowns, 1,000 sites with a
Gaussian well and four nonlocal projectors each, one 1,100-column block (the
benchmark's block for this workload).  The dense cell blocks R then hold
8,000 x 512 x 1,100 = 4.5e9 elements, past 2^31, so 64-bit offsets are
exercised in the cell kernel's stores and the assembly's reads.

The oracle applies H~ on sampled rows only (Eqs. discreteHam,
nonlocalHamDiscrete, hep): the cells holding each row, plus the projector
term C~^T h C~ X of the sites whose support reaches those cells.  Sites
farther than r_c + one cell diagonal from a sampled unknown contribute
exactly zero to its row and are left out of the oracle problem.  The rows sit
around the periodic corner node, which is shared by the first and the last
cells of the mesh, and next to the site at (2, 2, 2) bohr.
"""
import numpy as np
import pytest
import torch

from paper_1903_10959_gb300 import workloads as W

from gpu_util import gpu_context, rel_fro

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_c3_apply_sampled_rows_match_oracle():
    from oracle import hamiltonian as oham
    from oracle.fe import Mesh

    s = W.cubic_sites_nonlocal(block=1100)
    n1 = s.ncell * s.p
    M = n1 ** 3
    ncol = 1100
    ctx = gpu_context(s)
    try:
        assert ctx.ndofs == M
        ctx.set_blocking(ncol, 1)
        X = torch.empty((M, ncol), dtype=torch.float32, device=DEV)
        ctx.fill_uniform(X, s.seed, prec="bf16x3")
        Y = torch.empty_like(X)
        ctx.apply(X, Y, prec="bf16x3")

        def gidx(x, y, z):
            return (z * n1 + y) * n1 + x

        last = n1 - 1
        rows = np.array(sorted({gidx(0, 0, 0), gidx(3, 3, 3), gidx(0, 3, 5), gidx(last, last, last),
                                gidx(last, 0, 3), gidx(2, last, 0), gidx(7, 7, 7), gidx(9, 8, 7)}))
        cols = np.array([0, 1, 127, 128, 640, ncol - 1])
        got = Y[torch.as_tensor(rows, device=DEV)][:, torch.as_tensor(cols, device=DEV)]
        got = got.cpu().numpy().astype(np.float64)
        del X, Y
    finally:
        ctx.destroy()
    torch.cuda.empty_cache()

    # sites whose support can reach a cell holding a sampled unknown
    h = s.L / s.ncell
    xr = Mesh(s.ncell, s.p, s.L, True).dof_coords()[rows]
    d = xr[:, None, :] - s.nl_centres[None, :, :]
    d -= s.L * np.round(d / s.L)
    near = np.sqrt((d * d).sum(-1)).min(axis=0) <= s.nl_rcut + np.sqrt(3.0) * h + 1e-9
    sel = np.where(near)[0]
    assert 0 < len(sel) < len(s.nl_centres)
    prob = oham.wells_problem(s.ncell, s.p, s.L, True, s.centres, s.depths, s.widths,
                              projectors=dict(centres=s.nl_centres[sel], sigma=s.nl_sigma,
                                              rcut=s.nl_rcut, h=s.nl_h[sel]))
    # oracle input: the seeded block (binary32 rounding, as stored on the device)
    cnt = np.arange(M, dtype=np.uint64)[:, None] * np.uint64(ncol) + cols.astype(np.uint64)[None, :]
    X0 = W.uniform_pm1(s.seed, W.STREAM_X0, cnt).astype(np.float32).astype(np.float64)
    ref = prob.apply_Htilde_rows(rows, X0)
    # the projector term is present in these rows (not only the local part)
    assert abs(prob.C[:, rows]).sum() > 0
    assert rel_fro(got, ref) < 1e-5
    assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max()
