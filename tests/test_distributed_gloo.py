"""Partitioned ChFSI on CPU ranks (gloo): the domain split and the band split
of Sec. 3.7 against the unpartitioned oracle.

The partition (cells, local rows, owners, halo lists) is the library's host
logic (chfsi_partition_*); the communication and the order of the steps are
``paper_1903_10959_gb300.distributed``; each rank's arithmetic is the
oracle's, on its own rows (domain split: the cell loop over its cells,
``Problem.apply_Htilde_cells``) or its own columns (band split).

Checks: the partition covers every cell once and every unknown once as an
owner, and the halo lists agree pairwise; one H~ X (with and without
projectors, periodic, Dirichlet and semi-periodic meshes) equals the
unpartitioned oracle's rows to 1e-13; S and H^ all-reduced equal the
unpartitioned products; a whole ChFSI run gives the unpartitioned oracle's
eigenvalues to 1e-10 and the same subspace, on 2 and 4 ranks.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1903_10959_gb300 import workloads as W  # noqa: E402
from paper_1903_10959_gb300._lib import partition  # noqa: E402


# ----------------------------------------------------------------- host logic
MESHES = [(4, 10.0, 2, True), (3, 6.0, 3, False), (4, 8.0, 2, (True, True, False)),
          (5, 7.5, 2, (False, True, True))]


@pytest.mark.parametrize("mesh", MESHES)
@pytest.mark.parametrize("nranks", [1, 2, 3, 4, 6, 8])
def test_partition_covers_cells_and_unknowns(mesh, nranks):
    from oracle.fe import Mesh
    ncell, L, p, per = mesh
    om = Mesh(ncell, p, L, per)
    dm = om.dofmap()
    parts = [partition(ncell, L, p, per, nranks, r) for r in range(nranks)]
    cells = np.concatenate([P["cells"] for P in parts])
    assert np.array_equal(np.sort(cells), np.arange(om.ncells))
    owned = np.zeros(om.ndofs, np.int64)
    for r, P in enumerate(parts):
        # local rows = the unknowns of the rank's cells
        want = np.unique(dm[P["cells"]])
        want = want[want >= 0]
        assert np.array_equal(P["l2g"], want)
        np.add.at(owned, P["l2g"][P["owner"] == r], 1)
        assert np.all(P["owner"] <= r)              # the lowest rank touching a row owns it
        for q, h in zip(P["neighbors"], P["halo"]):
            Q = parts[q]
            k = list(Q["neighbors"]).index(r)
            # the shared rows: same unknowns, same order, on both sides
            assert np.array_equal(P["l2g"][h], Q["l2g"][Q["halo"][k]])
            both = np.intersect1d(want, np.unique(dm[Q["cells"]]))
            assert np.array_equal(P["l2g"][h], both[both >= 0])
    assert np.all(owned == 1)


def test_partition_rejects_too_many_ranks():
    from paper_1903_10959_gb300 import ChfsiError
    with pytest.raises(ChfsiError):
        partition(2, 4.0, 2, True, 16, 0)


# ----------------------------------------------------------------- rank workers
def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(fn, world, *args):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _port()
        procs = [ctx.Process(target=_worker, args=(fn, r, world, port, out) + args)
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(600)
        codes = [p.exitcode for p in procs]
        res = dict(out)
    assert codes == [0] * world, (codes, res.get("error"))
    return res


def _worker(fn, rank, world, port, out, *args):
    sys.path.insert(0, ROOT)
    import traceback

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = globals()[fn](rank, world, *args)
    except Exception:
        out["error"] = traceback.format_exc()
        raise
    finally:
        dist.destroy_process_group()


def _system(kind):
    if kind == "periodic":
        return W.small_periodic(seed=61, ncell=4, p=3, L=8.0, n_wells=4, n_want=12, degree=8, iters=3)
    if kind == "dirichlet":
        s = W.small_periodic(seed=62, ncell=4, p=3, L=8.0, n_wells=3, n_want=10, degree=8, iters=3)
        s.periodic = False
        s.centres = 0.1 * s.L + 0.8 * s.centres
        return s
    if kind == "slab":
        s = W.small_periodic(seed=63, ncell=4, p=3, L=8.0, n_wells=3, n_want=10, degree=8, iters=3)
        s.periodic = (True, True, False)
        return s
    # periodic with projectors
    s = W.cubic_sites_nonlocal(seed=64, ncell=4, p=3, L=8.0, n_side=2, n_want=12, degree=8, iters=3)
    return s


def _problem(s):
    from oracle import hamiltonian as oham
    proj = None
    if len(s.nl_centres):
        proj = dict(centres=s.nl_centres, sigma=s.nl_sigma, rcut=s.nl_rcut, h=s.nl_h)
    return oham.wells_problem(s.ncell, s.p, s.L, s.periodic, s.centres, s.depths, s.widths,
                              projectors=proj)


class _OracleDomain:
    """One rank's arithmetic in a domain split, from the oracle's formulas:
    the cell loop over the rank's cells (local part of Eq. hep), the projector
    coefficients C~ X from the owned rows and their expansion, and dense
    binary64 linear algebra on local rows."""

    def __init__(self, prob, ds):
        self.prob, self.ds = prob, ds
        self.s = prob.minv_sqrt
        if prob.C is not None:
            self.C = prob.C[:, ds.l2g].tocsr()
            self.Cown = prob.C[:, ds.l2g[ds.owned]].tocsr()

    def _T(self, a):
        import torch
        return torch.as_tensor(np.ascontiguousarray(a))

    def apply_partial(self, X):
        full = np.zeros((self.prob.ndofs, X.shape[1]))
        full[self.ds.l2g] = X.numpy()
        loc = self.prob.apply_Htilde_cells(self.ds.cells, full)
        return self._T(loc[self.ds.l2g])

    def nl_project(self, X):
        if self.prob.C is None:
            return None
        own = self.ds.owned
        return self._T(self.Cown @ (self.s[self.ds.l2g[own], None] * X.numpy()[own]))

    def nl_expand(self, Z, Y):
        e = self.s[self.ds.l2g, None] * (self.C.T @ (self.prob.hnl[:, None] * Z.numpy()))
        return Y + self._T(e)

    def recurrence(self, HY, Y, Yp, alpha, beta, c):
        out = alpha * (HY - c * Y)
        return out if Yp is None else out + beta * Yp

    def gram_owned(self, A, B):
        own = self.ds.owned
        return self._T(A.numpy()[own].T @ B.numpy()[own])

    def cholesky_inv_t(self, S):
        import scipy.linalg as sla
        L = np.linalg.cholesky(S.numpy())
        return self._T(sla.solve_triangular(L, np.eye(L.shape[0]), lower=True).T)

    def eigh(self, H):
        D, Q = np.linalg.eigh(H.numpy())
        return D, self._T(Q)

    def rotate(self, X, U):
        return self._T(X.numpy() @ U.numpy())


class _OracleBand:
    """One rank's arithmetic in a band split: the oracle's full H~ on its own
    columns and dense binary64 products over all rows."""

    def __init__(self, prob):
        self.prob = prob

    def _T(self, a):
        import torch
        return torch.as_tensor(np.ascontiguousarray(a))

    def apply(self, X):
        return self._T(self.prob.apply_Htilde(X.numpy()))

    def recurrence(self, HY, Y, Yp, alpha, beta, c):
        out = alpha * (HY - c * Y)
        return out if Yp is None else out + beta * Yp

    def gram(self, A, B):
        return self._T(A.numpy().T @ B.numpy())

    cholesky_inv_t = _OracleDomain.cholesky_inv_t
    eigh = _OracleDomain.eigh

    def rotate(self, X, U):
        return self._T(X.numpy() @ U.numpy())


def _domain_apply_job(rank, world, kind):
    import torch
    from paper_1903_10959_gb300 import distributed as D
    s = _system(kind)
    prob = _problem(s)
    ds = D.DomainSplit(s.ncell, s.L, s.p, s.periodic)
    be = _OracleDomain(prob, ds)
    X0 = W.start_block(s.seed, prob.ndofs, 5)
    Y = D.domain_apply(ds, be, torch.as_tensor(X0[ds.l2g]))
    Xl = torch.as_tensor(X0[ds.l2g])
    S = ds.allreduce(be.gram_owned(Xl, Xl))
    H = ds.allreduce(be.gram_owned(Xl, Y))
    return {"l2g": ds.l2g, "Y": Y.numpy(), "S": S.numpy(), "H": H.numpy(), "grid": ds.grid,
            "nbr": len(ds.neighbors)}


@pytest.mark.parametrize("kind", ["periodic", "dirichlet", "slab", "projectors"])
@pytest.mark.parametrize("world", [2, 4])
def test_domain_split_apply_and_panels(kind, world):
    s = _system(kind)
    prob = _problem(s)
    X0 = W.start_block(s.seed, prob.ndofs, 5)
    ref = prob.apply_Htilde(X0)
    res = _spawn("_domain_apply_job", world, kind)
    assert sum(res[r]["nbr"] for r in range(world)) > 0
    for r in range(world):
        got, l2g = res[r]["Y"], res[r]["l2g"]
        assert np.abs(got - ref[l2g]).max() <= 1e-13 * np.abs(ref).max()
        assert np.abs(res[r]["S"] - X0.T @ X0).max() <= 1e-13 * np.abs(X0.T @ X0).max()
        assert np.abs(res[r]["H"] - X0.T @ ref).max() <= 1e-12 * np.abs(X0.T @ ref).max()
    # shared rows hold the same bits on every rank that has them
    full = {}
    for r in range(world):
        for g, row in zip(res[r]["l2g"], res[r]["Y"]):
            if g in full:
                assert np.array_equal(full[g], row)
            full[g] = row
    assert len(full) == prob.ndofs


def _domain_chfsi_job(rank, world, kind, b):
    import torch
    from paper_1903_10959_gb300 import distributed as D
    s = _system(kind)
    prob = _problem(s)
    ds = D.DomainSplit(s.ncell, s.L, s.p, s.periodic)
    be = _OracleDomain(prob, ds)
    X0 = W.start_block(s.seed, prob.ndofs, s.n_sub)
    Dv, X = D.domain_chfsi(ds, be, torch.as_tensor(X0[ds.l2g]), s.degree, s.iters, b)
    return {"D": np.asarray(Dv), "X": X.numpy(), "l2g": ds.l2g}


def _band_chfsi_job(rank, world, kind, b):
    import torch
    from paper_1903_10959_gb300 import distributed as D
    s = _system(kind)
    prob = _problem(s)
    X0 = W.start_block(s.seed, prob.ndofs, s.n_sub)
    bs = D.BandSplit(s.n_sub)
    Dv, Xb = D.band_chfsi(bs, _OracleBand(prob), torch.as_tensor(X0[:, bs.c0:bs.c1]),
                          s.degree, s.iters, b)
    return {"D": np.asarray(Dv), "X": Xb.numpy(), "cols": (bs.c0, bs.c1)}


def _reference_chfsi(kind):
    from oracle import chfsi as och
    s = _system(kind)
    prob = _problem(s)
    b = och.lanczos_upper_bound(prob.apply_Htilde, W.lanczos_start(s.seed, prob.ndofs), 20)
    X0 = W.start_block(s.seed, prob.ndofs, s.n_sub)
    D, X = och.chfsi(prob.apply_Htilde, X0, s.degree, s.iters, b)
    return s, b, D, X


def _same_subspace(A, B):
    Pa = A @ np.linalg.solve(A.T @ A, A.T)
    Pb = B @ np.linalg.solve(B.T @ B, B.T)
    return np.linalg.norm(Pa - Pb)


@pytest.mark.parametrize("kind", ["periodic", "projectors"])
@pytest.mark.parametrize("world", [2, 4])
def test_domain_split_chfsi_matches_oracle(kind, world):
    s, b, D, X = _reference_chfsi(kind)
    res = _spawn("_domain_chfsi_job", world, kind, b)
    Xg = np.zeros_like(X)
    for r in range(world):
        assert np.abs(res[r]["D"] - D).max() <= 1e-10
        Xg[res[r]["l2g"]] = res[r]["X"]
    k = s.n_want
    assert _same_subspace(Xg[:, :k], X[:, :k]) <= 1e-8


@pytest.mark.parametrize("world", [2, 4])
def test_band_split_chfsi_matches_oracle(world):
    s, b, D, X = _reference_chfsi("periodic")
    res = _spawn("_band_chfsi_job", world, "periodic", b)
    Xg = np.zeros_like(X)
    for r in range(world):
        assert np.abs(res[r]["D"] - D).max() <= 1e-10
        c0, c1 = res[r]["cols"]
        Xg[:, c0:c1] = res[r]["X"]
    k = s.n_want
    assert _same_subspace(Xg[:, :k], X[:, :k]) <= 1e-8


def test_oracle_cell_subsets_sum_to_the_apply():
    """The oracle's per-subdomain cell loop summed over a partition of the
    cells is its full local apply (no projectors), to rounding."""
    s = _system("slab")
    prob = _problem(s)
    X = W.start_block(3, prob.ndofs, 3)
    rng = np.random.default_rng(5)
    lab = rng.integers(0, 3, prob.mesh.ncells)
    tot = sum(prob.apply_Htilde_cells(np.where(lab == k)[0], X) for k in range(3))
    ref = prob.apply_Htilde(X)
    assert np.abs(tot - ref).max() <= 1e-13 * np.abs(ref).max()
