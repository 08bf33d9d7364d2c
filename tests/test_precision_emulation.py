"""Numpy emulation of the mixed filter's arithmetic on the 4^3-cell, p = 4
workload (the residual-target analysis of the mixed path, and the reading
that FP16x2 products suffice).

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


def _f16(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float32)


def _pow2_scale(m):
    """2^(14 - E) for m = f 2^E, f in [0.5, 1): takes m into [2^13, 2^14)."""
    if not m > 0:
        return np.float32(1.0)
    return np.float32(np.ldexp(1.0, 14 - int(np.frexp(m)[1])))


def _split2(x):
    x = np.asarray(x, np.float32)
    t1 = _f16(x)
    return t1, _f16((x - t1).astype(np.float32))


def _f16x2_apply(prob):
    """Cell products as the FP16x2 kernel forms them: each cell matrix and each
    column of the block scaled by a power of two from its maximum, both split
    into two fp16 terms, the three kept products (h1 y2, h2 y1, h1 y1) summed
    in binary32, the scales undone exactly."""
    dm = prob.mesh.dofmap()
    s = prob.minv_sqrt
    cells = []
    for e, d in enumerate(dm):
        H = (s[d][:, None] * prob.cell_hamiltonian(e) * s[d][None, :]).astype(np.float32)
        se = _pow2_scale(np.abs(H).max())
        cells.append((_split2(H * se), se))
    order = ((0, 1), (1, 0), (0, 0))

    def apply(X):
        X32 = np.asarray(X, np.float32)
        out = np.zeros_like(X32)
        tc = np.array([_pow2_scale(v) for v in np.abs(X32).max(axis=0)], np.float32)
        for e, d in enumerate(dm):
            h, se = cells[e]
            y = _split2(X32[d] * tc[None, :])
            r = np.zeros((len(d), X32.shape[1]), np.float32)
            for i, j in order:
                r = (r + (h[i].astype(np.float64) @ y[j].astype(np.float64)).astype(np.float32)).astype(np.float32)
            np.add.at(out, d, (r / (se * tc[None, :])).astype(np.float32))
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


def test_f16x2_products_reach_the_same_binary32_floor():
    """Two fp16 terms per operand (about 22 bits, three products) leave the
    subspace at the floor the binary32 recurrence sets, as BF16x3's six
    products do: the generalized residual stalls in the same 1e-6 .. 3e-6
    band and the Ritz values agree with the BF16x3-emulated run to 1e-10 Ha
    (the cell products are not what limits the binary32 filter)."""
    sy = W.small_periodic()
    prob = oham.wells_problem(sy.ncell, sy.p, sy.L, True, sy.centres, sy.depths, sy.widths)
    Ht = prob.apply_Htilde
    b = och.lanczos_upper_bound(Ht, W.lanczos_start(sy.seed, prob.ndofs), 20)
    out = []
    for apply in (_f16x2_apply(prob), _bf16x3_apply(prob)):
        X = och.cholgs(W.start_block(sy.seed, prob.ndofs, sy.n_sub))
        D, X = och.rayleigh_ritz(Ht, X)
        for _ in range(2 * sy.iters):
            X = och.cholgs(_filter32(apply, X, sy.degree, D[-1], b, D[0]))
            D, X = och.rayleigh_ritz(Ht, X)
        n = sy.n_want
        out.append((D[:n], och.generalized_residual_norms(Ht, X, D, prob.mass)[:n].max()))
    (d16, f16), (dbf, fbf) = out
    assert 1e-6 < f16 < 3e-6 and 1e-6 < fbf < 3e-6
    assert np.abs(d16 - dbf).max() < 1e-10


def test_f16x2_split_error_bound():
    """The split itself: for values scaled into [2^13, 2^14) by their maximum,
    two fp16 terms hold each binary32 value to 2^-22 of the maximum, and the
    three kept products of a dot product stay within 2^-21 of sum |a||y|."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        a = (rng.standard_normal(343) * np.exp(rng.uniform(-8, 8))).astype(np.float32)
        y = (rng.standard_normal(343) * np.exp(rng.uniform(-8, 8))).astype(np.float32)
        sa, sy = _pow2_scale(np.abs(a).max()), _pow2_scale(np.abs(y).max())
        assert 2.0 ** 13 <= np.abs(a * sa).max() < 2.0 ** 14
        a1, a2 = _split2(a * sa)
        y1, y2 = _split2(y * sy)
        rep = (a1.astype(np.float64) + a2) / sa
        assert np.abs(rep - a).max() <= 2.0 ** -22 * np.abs(a).max()
        got = (np.dot(a1.astype(np.float64), y2) + np.dot(a2.astype(np.float64), y1)
               + np.dot(a1.astype(np.float64), y1)) / (sa * sy)
        exact = np.dot(a.astype(np.float64), y.astype(np.float64))
        assert abs(got - exact) <= 2.0 ** -21 * np.dot(np.abs(a.astype(np.float64)), np.abs(y))
