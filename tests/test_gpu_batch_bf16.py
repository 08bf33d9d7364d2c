"""Batched BF16x3 filtering and ChFSI: per Chebyshev degree step one launch of
the BF16x3 cell kernel over the (system, cell, 128-column tile, row part)
items of every system and one launch of the batched assembly.

References: the single-system BF16x3 filter (the same per-item arithmetic;
1e-6 relative because the batch keeps the recurrence scalars in binary32),
the FP64 oracle filter (1e-4, as for the other mixed precisions) and the
oracle's ChFSI eigenvalues (the method statement's 1e-7 Ha, converged pairs).
Cases cover one row part (p = 5) and two (p = 6, 7), block widths below one
128-column tile, ragged and several tiles, Dirichlet and periodic members.
"""
import numpy as np
import pytest
import torch

from paper_1903_10959_gb300 import Batch, ChfsiError, workloads as W
from oracle import chfsi as och

from gpu_util import gpu_context, oracle_problem, rel_fro

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _members(p, shapes, periodic=False):
    out = []
    for k, (n, nw) in enumerate(shapes):
        s = W.small_periodic(seed=60 + 7 * p + k, ncell=n, p=p, L=1.6 * n, n_wells=nw, n_want=10,
                             degree=10, iters=5)
        if not periodic:
            s.periodic = False
            s.centres = 0.1 * s.L + 0.8 * s.centres
        out.append(s)
    return out


def _filter_case(systems, widths, degree, seed0):
    ctxs = [gpu_context(s) for s in systems]
    try:
        probs = [oracle_problem(s) for s in systems]
        X0 = [W.start_block(seed0 + i, c.ndofs, w).astype(np.float32)
              for i, (c, w) in enumerate(zip(ctxs, widths))]
        b = np.array([och.lanczos_upper_bound(p.apply_Htilde, W.lanczos_start(3, p.ndofs), 15)
                      for p in probs])
        a, a0 = 0.2 * b, np.full(len(b), -3.0)
        B = Batch(ctxs)
        X = [torch.tensor(x, device=DEV) for x in X0]
        B.filter(X, degree, a, b, a0, prec="bf16x3")
        for i, (c, p) in enumerate(zip(ctxs, probs)):
            Xs = torch.tensor(X0[i], device=DEV)
            c.filter(Xs, degree, a[i], b[i], a0[i], prec="bf16x3")
            got = X[i].cpu().numpy()
            assert np.isfinite(got).all()
            assert rel_fro(got, Xs.cpu().numpy()) < 1e-6, i
            ref = och.chebyshev_filter(p.apply_Htilde, X0[i].astype(np.float64), degree, a[i], b[i], a0[i])
            assert rel_fro(got.astype(np.float64), ref) < 1e-4, i
        B.destroy()
    finally:
        for c in ctxs:
            c.destroy()


def test_one_part_ragged_and_several_tiles():
    # p = 5: n_e = 216, one row part; widths 5 (< one tile), 130 (ragged), 257 (three tiles)
    systems = _members(5, [(2, 3), (3, 4), (3, 5), (2, 2)])
    _filter_case(systems, [5, 130, 257, 20], 10, 11)


@pytest.mark.parametrize("p", [6, 7])
def test_two_parts(p):
    # p = 6 (n_e = 343) and p = 7 (n_e = 512): two row parts per cell
    systems = _members(p, [(2, 3), (2, 4), (2, 2)])
    _filter_case(systems, [7, 140, 64], 8, 21)


def test_periodic_members():
    systems = _members(4, [(3, 3), (2, 2)], periodic=True)
    _filter_case(systems, [33, 129], 9, 31)


def test_precision_switch_recaptures_and_autotune_refuses():
    systems = _members(5, [(2, 3), (3, 4)])
    ctxs = [gpu_context(s) for s in systems]
    try:
        B = Batch(ctxs)
        X0 = [W.start_block(41 + i, c.ndofs, 40).astype(np.float32) for i, c in enumerate(ctxs)]
        n = len(ctxs)
        a, b, a0 = np.full(n, 5.0), np.full(n, 60.0), np.full(n, -3.0)
        out = {}
        for prec in ("mixed", "bf16x3", "mixed", "bf16x3"):
            X = [torch.tensor(x, device=DEV) for x in X0]
            B.filter(X, 6, a, b, a0, prec=prec)
            got = [x.cpu().numpy() for x in X]
            if prec in out:                              # a replay equals the first capture
                assert all(np.array_equal(g, o) for g, o in zip(got, out[prec]))
            out[prec] = got
        for i, c in enumerate(ctxs):
            Xs = torch.tensor(X0[i], device=DEV)
            c.filter(Xs, 6, 5.0, 60.0, -3.0, prec="bf16x3")
            assert rel_fro(out["bf16x3"][i], Xs.cpu().numpy()) < 1e-6
        with pytest.raises(ChfsiError):
            B.autotune([torch.tensor(x, device=DEV) for x in X0], prec="bf16x3")
        B.destroy()
    finally:
        for c in ctxs:
            c.destroy()


def test_batched_solve_bf16x3_filter_and_orthogonalisation():
    systems = _members(5, [(2, 3), (3, 5), (3, 2)])
    ctxs = [gpu_context(s) for s in systems]
    try:
        probs = [oracle_problem(s) for s in systems]
        bnd = np.array([och.lanczos_upper_bound(p.apply_Htilde, W.lanczos_start(4, p.ndofs), 15)
                        for p in probs])
        iters, m = 14, 12
        X0 = [W.start_block(s.seed, c.ndofs, s.n_sub) for s, c in zip(systems, ctxs)]
        B = Batch(ctxs)
        X = [torch.tensor(x, device=DEV) for x in X0]
        evs = B.solve(X, iters, m, bnd, filter_prec="bf16x3", orth_prec="bf16x3")
        B.destroy()
        for i, (s, p) in enumerate(zip(systems, probs)):
            D_ref, _ = och.chfsi(p.apply_Htilde, X0[i], m, iters, bnd[i])
            assert np.abs(evs[i][:s.n_want] - D_ref[:s.n_want]).max() < 1e-7
            Q = X[i].cpu().numpy()
            assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-4
    finally:
        for c in ctxs:
            c.destroy()
