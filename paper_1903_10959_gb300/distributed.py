"""Partitioned ChFSI over several ranks: the two levels of parallelism of
Sec. 3.7 of arXiv:1903.10959.

Domain split (the primary level): each rank owns a block of cells
(``chfsi_partition_*``) and the rows of X at the unknowns its cells touch.
One H~ X is the rank's cell loop (partial sums on its rows) completed by a
halo sum: every rank sends its partial sums on the unknowns shared with a
neighbour and adds what the neighbours send; shared rows are summed in
ascending rank order, so every rank holding a shared row ends with the same
bits.  The projector term needs the projected coefficients Z = C~ X summed
over all ranks (each unknown counted by its owner) before the expansion.
The overlap S = X^T X (Algorithm CholGS step 1) and the projected matrix
H^ = X^T H~ X (Sec. 3.5) are sums over the owned rows, completed by an
all-reduce of the N x N panels (the paper's blocked MPI_Allreduce of S);
the factorisations are then repeated on every rank, and the rotations
X <- X U act on local rows only.

Band split (the second level): each rank holds all rows and a contiguous
group of columns.  The filter needs no communication (Sec. 3.7: each
wavefunction is filtered independently).  CholGS gathers the block, forms
its own columns S_b = X^T X_b, gathers S, factors it on every rank and keeps
X_b <- X L^{-T}_b (the N x N_b columns of L^{-T}); Rayleigh-Ritz likewise
with H^_b = X^T H~ X_b and X_b <- X Q_b.

This module holds the communication and the order of the steps only.  All
arithmetic is the backend's (``DomainBackend`` / ``BandBackend`` below): on
GPUs each rank's backend is the library's kernels on its local rows, with
the collectives on NCCL (halo rows sent and received into the rank's own
device memory; no cross-GPU multicast); the CPU emulation of the tests uses
gloo and the oracle's arithmetic.
"""
from __future__ import annotations

from typing import Protocol

from ._lib import partition


def _dist():
    import torch.distributed as dist
    return dist


# --------------------------------------------------------------------- domain split
class DomainSplit:
    """One rank's share of a domain decomposition of the mesh.

    ``l2g``: global unknowns of the rank's rows (ascending), ``owned``: mask
    of the rows the rank counts in sums over unknowns, ``halo[k]``: local rows
    shared with ``neighbors[k]`` (ascending global order, identical on both
    sides)."""

    def __init__(self, ncell, length, p, periodic, group=None):
        dist = _dist()
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        part = partition(ncell, length, p, periodic, self.world, self.rank)
        self.cells = part["cells"]
        self.l2g = part["l2g"]
        self.owned = part["owner"] == self.rank
        self.neighbors = [int(q) for q in part["neighbors"]]
        self.halo = part["halo"]
        self.grid = part["grid"]
        self._global_rank = [dist.get_global_rank(group, q) if group is not None else q
                             for q in range(self.world)]

    @property
    def nlocal(self):
        return len(self.l2g)

    def halo_sum(self, Y):
        """Complete the partial sums Y (nlocal x k torch tensor, CPU or CUDA)
        on the shared rows; returns a new tensor."""
        import torch
        dist = _dist()
        if not self.neighbors:
            return Y
        idx = [torch.as_tensor(h, dtype=torch.long, device=Y.device) for h in self.halo]
        sends = [Y.index_select(0, i).contiguous() for i in idx]
        recvs = [torch.empty_like(sb) for sb in sends]
        ops = []
        for q, sb, rb in zip(self.neighbors, sends, recvs):
            g = self._global_rank[q]
            ops.append(dist.P2POp(dist.isend, sb, g, self.group))
            ops.append(dist.P2POp(dist.irecv, rb, g, self.group))
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        # ascending rank order over {me} U neighbours: every sharer of a row adds
        # the same partial sums in the same order
        out = torch.zeros_like(Y)
        order = sorted([(self.rank, None)] + list(zip(self.neighbors, range(len(self.neighbors)))))
        for q, k in order:
            if k is None:
                out += Y
            else:
                out.index_add_(0, idx[k], recvs[k])
        return out

    def allreduce(self, T):
        _dist().all_reduce(T, op=_dist().ReduceOp.SUM, group=self.group)
        return T


class DomainBackend(Protocol):
    """Arithmetic of one rank in a domain split (local rows, local numbering)."""

    def apply_partial(self, X): ...        # sum over own cells of H~_e X_e (partial sums)

    def nl_project(self, X): ...           # projector coefficients from owned rows, or None

    def nl_expand(self, Z, Y): ...         # Y + C~^T h Z on local rows

    def recurrence(self, HY, Y, Yprev, alpha, beta, shift): ...   # alpha (HY - shift Y) + beta Yprev

    def gram_owned(self, A, B): ...        # A^T B over the owned rows

    def cholesky_inv_t(self, S): ...       # U = L^{-T}, S = L L^T

    def eigh(self, H): ...                 # ascending (D, Q)

    def rotate(self, X, U): ...            # X U on local rows


def domain_apply(ds: DomainSplit, be: DomainBackend, X):
    """Rows l2g of H~ X (Eq. hep): cell loop, halo sum, projector term."""
    Y = ds.halo_sum(be.apply_partial(X))
    Z = be.nl_project(X)
    if Z is not None:
        Y = be.nl_expand(ds.allreduce(Z), Y)
    return Y


def filter_steps(m, a, b, a0):
    """(alpha_k, beta_k) of the scaled recurrence (Eq. chebFilter, Zhou-Saad form)
    and the shift c: Y_k = alpha_k (H~ Y_{k-1} - c Y_{k-1}) + beta_k Y_{k-2}."""
    e, c = (b - a) / 2.0, (b + a) / 2.0
    s1 = e / (a0 - c)
    out, s = [(s1 / e, 0.0)], s1
    for _ in range(2, m + 1):
        sn = 1.0 / (2.0 / s1 - s)
        out.append((2.0 * sn / e, -s * sn))
        s = sn
    return out, c


def domain_filter(ds, be, X, m, a, b, a0):
    steps, c = filter_steps(m, a, b, a0)
    Yp, Y = None, X
    for alpha, beta in steps:
        Yn = be.recurrence(domain_apply(ds, be, Y), Y, Yp, alpha, beta, c)
        Yp, Y = Y, Yn
    return Y


def domain_cholgs(ds, be, X):
    """Algorithm CholGS on row-distributed X: S all-reduced, X <- X L^{-T}."""
    S = ds.allreduce(be.gram_owned(X, X))
    return be.rotate(X, be.cholesky_inv_t(S))


def domain_rayleigh_ritz(ds, be, X):
    """Sec. 3.5 on row-distributed X: H^ all-reduced, H^ Q = Q D, X <- X Q."""
    H = ds.allreduce(be.gram_owned(X, domain_apply(ds, be, X)))
    D, Q = be.eigh(H)
    return D, be.rotate(X, Q)


def domain_chfsi(ds, be, X, m, iters, b):
    """The ChFSI loop (step 7 of Algorithm scf, repeated) on a domain split."""
    X = domain_cholgs(ds, be, X)
    D, X = domain_rayleigh_ritz(ds, be, X)
    for _ in range(iters):
        X = domain_filter(ds, be, X, m, float(D[-1]), b, float(D[0]))
        X = domain_cholgs(ds, be, X)
        D, X = domain_rayleigh_ritz(ds, be, X)
    return D, X


# --------------------------------------------------------------------- band split
class BandSplit:
    """Column groups of a band split: rank r holds columns [c0, c1) of N."""

    def __init__(self, ncols, group=None):
        dist = _dist()
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.n = ncols
        self.bounds = [(q * ncols // self.world, (q + 1) * ncols // self.world)
                       for q in range(self.world)]
        self.c0, self.c1 = self.bounds[self.rank]

    def gather_columns(self, Xb):
        """All groups' columns side by side (rows x N), in group order."""
        import torch
        dist = _dist()
        w = max(c1 - c0 for c0, c1 in self.bounds)
        pad = torch.zeros((Xb.shape[0], w), dtype=Xb.dtype, device=Xb.device)
        pad[:, :Xb.shape[1]] = Xb
        parts = [torch.empty_like(pad) for _ in range(self.world)]
        dist.all_gather(parts, pad, group=self.group)
        return torch.cat([parts[q][:, :c1 - c0] for q, (c0, c1) in enumerate(self.bounds)], dim=1)


class BandBackend(Protocol):
    """Arithmetic of one rank in a band split (all rows, own columns)."""

    def apply(self, X): ...                # H~ X

    def recurrence(self, HY, Y, Yprev, alpha, beta, shift): ...

    def gram(self, A, B): ...              # A^T B over all rows

    def cholesky_inv_t(self, S): ...

    def eigh(self, H): ...

    def rotate(self, X, U): ...


def band_filter(bs, be, Xb, m, a, b, a0):
    """Chebyshev filter of the rank's own columns: no communication."""
    steps, c = filter_steps(m, a, b, a0)
    Yp, Y = None, Xb
    for alpha, beta in steps:
        Yn = be.recurrence(be.apply(Y), Y, Yp, alpha, beta, c)
        Yp, Y = Y, Yn
    return Y


def band_cholgs(bs, be, Xb):
    X = bs.gather_columns(Xb)
    S = bs.gather_columns(be.gram(X, Xb))                 # S_b = X^T X_b, then all of S
    U = be.cholesky_inv_t(S)
    return be.rotate(X, U[:, bs.c0:bs.c1].contiguous())


def band_rayleigh_ritz(bs, be, Xb):
    X = bs.gather_columns(Xb)
    H = bs.gather_columns(be.gram(X, be.apply(Xb)))       # H^_b = X^T H~ X_b
    D, Q = be.eigh(H)
    return D, be.rotate(X, Q[:, bs.c0:bs.c1].contiguous())


def band_chfsi(bs, be, Xb, m, iters, b):
    Xb = band_cholgs(bs, be, Xb)
    D, Xb = band_rayleigh_ritz(bs, be, Xb)
    for _ in range(iters):
        Xb = band_filter(bs, be, Xb, m, float(D[-1]), b, float(D[0]))
        Xb = band_cholgs(bs, be, Xb)
        D, Xb = band_rayleigh_ritz(bs, be, Xb)
    return D, Xb
