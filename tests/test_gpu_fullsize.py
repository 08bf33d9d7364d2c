"""Parity at the benchmark's full size: the 16^3-cell p = 6 FCC system
(884,736 unknowns, 1,100 columns) in the launch configuration the benchmark
times (all columns in one block; BF16x3 cell products, the default, and
3xTF32).

The oracle cannot apply H~ to the whole block, so one application is checked
on sampled rows and columns (the oracle sums only the cells holding each
sampled unknown), and a degree-3 filter on sampled rows of sampled columns:
row j of Y_k depends only on the rows of Y_{k-1} in the cells holding j, so
the oracle's own filter (Eq. chebFilter) driven by an apply that evaluates
the two-cell-layer neighbourhood of the sampled rows gives those rows
exactly.  CholGS and Rayleigh-Ritz are checked through properties that hold
at any size: column independence of the filter (bit-identical whether a
column is filtered with the whole block or alone), orthonormality after
CholGS, and Ritz values equal to the Rayleigh quotients of the rotated block.
"""
import numpy as np
import pytest
import torch

from oracle import chfsi as och
from paper_1903_10959_gb300 import workloads as W

from gpu_util import gpu_context, oracle_problem, rel_fro

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def full():
    s = W.fcc_periodic()
    ctx = gpu_context(s)
    n = s.n_sub
    ctx.set_blocking(n, 1)           # one block of all columns (the benchmark's choice)
    ctx.set_cell_tile(64)
    X = torch.empty((ctx.ndofs, n), dtype=torch.float32, device=DEV)
    ctx.fill_uniform(X, s.seed, prec="mixed")
    yield s, ctx, X
    ctx.destroy()


@pytest.fixture(scope="module")
def oprob():
    """The oracle problem of the same system (cell matrices cached as used)."""
    return oracle_problem(W.fcc_periodic())


def _sample(s, M, rng_seed=7):
    """Sampled unknowns: interior nodes of a few cells and nodes shared by
    2, 4 and 8 cells (face, edge, corner), plus the last unknown."""
    n1 = s.ncell * s.p
    pts = [(3, 3, 3), (0, 4, 5), (0, 0, 2), (0, 0, 0), (n1 - 1, n1 - 1, n1 - 1), (17, 50, 6),
           (6, 6, 90), (48, 48, 48), (1, 60, 95), (95, 0, 37)]
    rows = [(i * n1 + j) * n1 + k for k, j, i in pts] + [M - 1]
    return np.array(sorted(set(rows)), dtype=np.int64)


def test_fill_matches_generator(full):
    s, ctx, X = full
    rows = _sample(s, ctx.ndofs)
    host = W.start_block(s.seed, rows, s.n_sub).astype(np.float32)
    assert np.array_equal(X[torch.as_tensor(rows, device=DEV)].cpu().numpy(), host)


def _x0_columns(s, M, cols):
    """Columns `cols` of the seeded start block, rounded to binary32 like the
    device copy, as binary64 oracle input."""
    cnt = np.arange(M, dtype=np.uint64)[:, None] * np.uint64(s.n_sub) + cols.astype(np.uint64)[None, :]
    return W.uniform_pm1(s.seed, W.STREAM_X0, cnt).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "f16x2"])
def test_apply_sampled_rows_match_oracle(full, oprob, prec):
    s, ctx, X = full
    M, n = ctx.ndofs, s.n_sub
    Y = torch.empty_like(X)
    ctx.apply(X, Y, prec=prec)
    rows = _sample(s, M)
    cols = np.array([0, 1, 63, 64, 127, 500, 511, 512, 1000, n - 1])
    X0 = _x0_columns(s, M, cols)
    prob = oprob
    ref = prob.apply_Htilde_rows(rows, X0)
    got = Y[torch.as_tensor(rows, device=DEV)][:, torch.as_tensor(cols, device=DEV)]
    got = got.cpu().numpy().astype(np.float64)
    assert rel_fro(got, ref) < 1e-5
    # per element, against the size of the row's terms (3xTF32: ~2^-22 per
    # product; BF16x3 drops only terms below 2^-23 of each product)
    assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["bf16x3", "f16x2"])
def test_filter_sampled_rows_match_oracle(full, oprob, prec):
    """Degree-3 BF16x3 filter of the whole 1,100-column block (the bench's
    block and kernel) against the oracle filter of four of its columns, on
    unknowns of one cell: interior, face, edge and corner nodes."""
    s, ctx, X = full
    M, n = ctx.ndofs, s.n_sub
    a, b, a0, m = 5.0, 2000.0, -3.0, 3
    Xf = X.clone()
    ctx.filter(Xf, m, a, b, a0, prec=prec)
    n1 = s.ncell * s.p

    def gidx(x, y, z):
        return (z * n1 + y) * n1 + x

    rows = np.array(sorted({gidx(33, 33, 33), gidx(30, 33, 33), gidx(30, 30, 33),
                            gidx(30, 30, 30), gidx(31, 35, 34)}))
    cols = np.array([0, 127, 128, n - 1])
    prob = oprob
    dm = prob.mesh.dofmap()

    def stencil(r):        # unknowns of every cell holding one of the rows r
        return np.unique(dm[np.isin(dm, r).any(axis=1)])

    near = stencil(stencil(rows))          # rows of Y_1 that Y_3's rows depend on

    def local_apply(Y):
        out = np.zeros_like(Y)
        out[near] = prob.apply_Htilde_rows(near, Y)
        return out

    ref = och.chebyshev_filter(local_apply, _x0_columns(s, M, cols), m, a, b, a0)[rows]
    got = Xf[torch.as_tensor(rows, device=DEV)][:, torch.as_tensor(cols, device=DEV)]
    got = got.cpu().numpy().astype(np.float64)
    assert rel_fro(got, ref) < 1e-4
    del Xf


def test_filter_column_independent_of_block(full):
    """A column filtered with all 1,100 columns equals the same column filtered
    alone (another grid, another tile shape, same arithmetic per element)."""
    s, ctx, X = full
    cols = [0, 77, 700, s.n_sub - 1]
    Xb = X.clone()
    Xs = X[:, cols].contiguous()
    ctx.filter(Xb, 6, 20.0, 300.0, -1.0, prec="mixed")
    ctx.set_blocking(8, 1)
    ctx.filter(Xs, 6, 20.0, 300.0, -1.0, prec="mixed")
    ctx.set_blocking(s.n_sub, 1)
    assert torch.equal(Xb[:, cols], Xs)


def test_cholgs_and_rr_at_full_size(full):
    s, ctx, X = full
    n = s.n_sub
    Q = X.clone()
    ctx.cholgs(Q, prec="mixed")
    q64 = Q.double()
    G = q64.T @ q64
    assert (G - torch.eye(n, device=DEV, dtype=torch.float64)).abs().max().item() < 5e-5
    D = ctx.rayleigh_ritz(Q, prec="mixed")
    assert np.all(np.diff(D) >= 0)
    # Ritz values = Rayleigh quotients of the rotated block, H~ applied in binary64
    sel = [0, 1, n // 2, n - 1]
    Z = Q[:, sel].double().contiguous()
    HZ = torch.empty_like(Z)
    ctx.apply(Z, HZ, prec="fp64")
    rq = ((Z * HZ).sum(0) / (Z * Z).sum(0)).cpu().numpy()
    assert np.abs(rq - D[sel]).max() < 1e-4 * max(1.0, np.abs(D).max())
    del q64, G, Z, HZ
