"""Numpy emulation of the mixed filter's arithmetic on the 4^3-cell, p = 4
workload (the residual-target analysis of the mixed path).

The cell products are emulated as BF16x3 (both operands split into three bf16
terms, the six kept cross products summed in binary32), the recurrence and
the assembly are stored and accumulated in binary32, and CholGS / RR run in
binary64 (the oracle).  This pins two facts the mixed path's precision
reading rests on: such a binary32-filtered subspace stalls with a generalized
residual between 1e-6 and 3e-6, and one binary64 filter / CholGS / RR pass
after it brings the residual under 1e-6, also after the block is stored back
in binary32."""
import numpy as np

from oracle import chfsi as och
from oracle import hamiltonian as oham
from paper_1903_10959_gb300 import workloads as W


def _bf16(x):
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _split3(x):
    x = np.asarray(x, np.float32)
    t1 = _bf16(x)
    r1 = (x - t1).astype(np.float32)
    t2 = _bf16(r1)
    return t1, t2, _bf16((r1 - t2).astype(np.float32))


def _bf16x3_apply(prob):
    dm = prob.mesh.dofmap()
    s = prob.minv_sqrt
    cells = [_split3(s[d][:, None] * prob.cell_hamiltonian(e) * s[d][None, :])
             for e, d in enumerate(dm)]
    order = ((2, 0), (1, 1), (0, 2), (1, 0), (0, 1), (0, 0))      # smallest products first

    def apply(X):
        X32 = np.asarray(X, np.float32)
        out = np.zeros_like(X32)
        for e, d in enumerate(dm):
            h, y = cells[e], _split3(X32[d])
            r = np.zeros((len(d), X32.shape[1]), np.float32)
            for i, j in order:
                r = (r + (h[i].astype(np.float64) @ y[j].astype(np.float64)).astype(np.float32)).astype(np.float32)
            np.add.at(out, d, r)
        return out
    return apply


def _filter32(apply, X, m, a, b, a0):
    """Scaled Chebyshev recurrence (Eq. chebFilter, Zhou-Saad form) in binary32."""
    e, c = (b - a) / 2, (b + a) / 2
    s1 = e / (a0 - c)
    s = s1
    Yp = X.astype(np.float32)
    Y = (np.float32(s1 / e) * (apply(Yp) - np.float32(c) * Yp)).astype(np.float32)
    for _ in range(2, m + 1):
        sn = 1.0 / (2.0 / s1 - s)
        Yn = (np.float32(2 * sn / e) * (apply(Y) - np.float32(c) * Y) - np.float32(s * sn) * Yp).astype(np.float32)
        Yp, Y, s = Y, Yn, sn
    return Y.astype(np.float64)


def test_binary32_floor_and_binary64_polish():
    sy = W.small_periodic()
    prob = oham.wells_problem(sy.ncell, sy.p, sy.L, True, sy.centres, sy.depths, sy.widths)
    Ht = prob.apply_Htilde
    b = och.lanczos_upper_bound(Ht, W.lanczos_start(sy.seed, prob.ndofs), 20)
    apply = _bf16x3_apply(prob)
    X = och.cholgs(W.start_block(sy.seed, prob.ndofs, sy.n_sub))
    D, X = och.rayleigh_ritz(Ht, X)
    for _ in range(2 * sy.iters):
        X = och.cholgs(_filter32(apply, X, sy.degree, D[-1], b, D[0]))
        D, X = och.rayleigh_ritz(Ht, X)
    n = sy.n_want
    floor = och.generalized_residual_norms(Ht, X, D, prob.mass)[:n].max()
    assert 1e-6 < floor < 3e-6
    X = och.cholgs(och.chebyshev_filter(Ht, X, 8, D[-1], b, D[0]))
    D, X = och.rayleigh_ritz(Ht, X)
    polished = och.generalized_residual_norms(Ht, X, D, prob.mass)[:n].max()
    stored = och.generalized_residual_norms(Ht, X.astype(np.float32).astype(np.float64), D, prob.mass)[:n].max()
    assert polished < 1e-6 and stored < 1e-6 and polished < floor
