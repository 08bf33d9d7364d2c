"""Seeded synthetic inputs for the ChFSI workloads.

This module only draws random numbers and lays out problem descriptions; it
holds none of the method's arithmetic (no basis functions, no Hamiltonian, no
filter).  Both the CUDA path and the FP64 CPU checker read the arrays it
produces, so they always see the same inputs.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw ``i`` of stream ``(seed, stream)`` is the SplitMix64 output
for state ``key(seed, stream) + (i + 1) * GOLDEN``.  The device fill kernel of
the library implements the same published definition, so large start blocks
can be generated on the GPU and sampled rows regenerated here.

Workload shapes follow the paper's pseudopotential benchmarks (periodic metal
supercells, Chebyshev degree 20-50, Sec. 3.3 and Table 7); the atoms are
replaced by attractive Gaussian wells and optional Gaussian projectors.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)

# stream identifiers (one per kind of array)
STREAM_X0 = 1
STREAM_CENTRES = 2
STREAM_DEPTHS = 3
STREAM_WIDTHS = 4
STREAM_JITTER = 5
STREAM_NL_H = 6
STREAM_LANCZOS = 7
STREAM_SYSTEMS = 8
STREAM_NOISE = 9


def _finalize(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of stream ``stream`` under ``seed``: finalize(seed) xor stream*C."""
    with np.errstate(over="ignore"):
        k = _finalize(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)]))[0]
        return np.uint64(k ^ (np.uint64(stream) * _STREAM_MUL))


def raw_u64(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 outputs for the given draw counters (uint64 array)."""
    key = stream_key(seed, stream)
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = key + (c + np.uint64(1)) * GOLDEN
    return _finalize(state)


def uniform01(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of the SplitMix64 output."""
    r = raw_u64(seed, stream, counters) >> np.uint64(11)
    return r.astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_pm1(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [-1, 1): 2u - 1 (exact in binary64)."""
    return 2.0 * uniform01(seed, stream, counters) - 1.0


def start_block(seed: int, rows: np.ndarray | int, ncols: int) -> np.ndarray:
    """Rows of the seeded start block X0 (M x ncols, row-major).

    Element (r, c) is draw ``r * ncols + c`` of stream STREAM_X0, mapped to
    [-1, 1).  ``rows`` is either a row count (all rows 0..rows-1) or an index
    array of sampled rows.
    """
    if np.isscalar(rows):
        rows = np.arange(int(rows), dtype=np.uint64)
    rows = np.asarray(rows, dtype=np.uint64)
    cnt = rows[:, None] * np.uint64(ncols) + np.arange(ncols, dtype=np.uint64)[None, :]
    return uniform_pm1(seed, STREAM_X0, cnt)


def lanczos_start(seed: int, m: int) -> np.ndarray:
    """Seeded start vector of the Lanczos bound estimate (length m)."""
    return uniform_pm1(seed, STREAM_LANCZOS, np.arange(m, dtype=np.uint64))


@dataclass
class System:
    """One synthetic eigenproblem: mesh, wells, projectors, solver settings."""

    name: str
    ncell: int                  # cells per side (cubic box)
    p: int                      # FE degree
    L: float                    # box side (bohr)
    periodic: bool
    centres: np.ndarray         # (n_wells, 3)
    depths: np.ndarray          # (n_wells,), well depth D_a > 0 (V = -D exp(..))
    widths: np.ndarray          # (n_wells,)
    n_want: int                 # eigenpairs requested
    degree: int                 # Chebyshev degree m
    iters: int
    seed: int
    block: int = 0              # column block of the filter (0: all columns)
    nl_centres: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    nl_sigma: float = 0.8
    nl_rcut: float = 3.0
    nl_h: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))

    @property
    def n_nodes_1d(self) -> int:
        return self.ncell * self.p if self.periodic else self.ncell * self.p - 1

    @property
    def ndofs(self) -> int:
        return self.n_nodes_1d ** 3

    @property
    def n_buffer(self) -> int:
        return max(4, math.ceil(0.1 * self.n_want))

    @property
    def n_sub(self) -> int:
        """Subspace size: requested pairs plus a 10 % (at least 4) buffer."""
        return self.n_want + self.n_buffer


def _wells_uniform(seed: int, n: int, lo: np.ndarray, hi: np.ndarray):
    cnt = np.arange(3 * n, dtype=np.uint64)
    u = uniform01(seed, STREAM_CENTRES, cnt).reshape(n, 3)
    centres = lo + (hi - lo) * u
    depths = 1.0 + 2.0 * uniform01(seed, STREAM_DEPTHS, np.arange(n, dtype=np.uint64))
    widths = 0.8 + 0.4 * uniform01(seed, STREAM_WIDTHS, np.arange(n, dtype=np.uint64))
    return centres, depths, widths


def small_periodic(seed: int = 1, ncell: int = 4, p: int = 4, L: float = 10.0,
                   n_wells: int = 8, n_want: int = 32, degree: int = 20,
                   iters: int = 10) -> System:
    """Periodic box, wells at uniform random centres (4^3 cells, p=4 default)."""
    c, d, w = _wells_uniform(seed, n_wells, np.zeros(3), np.full(3, L))
    return System("periodic-%dc-p%d" % (ncell, p), ncell, p, L, True, c, d, w,
                  n_want, degree, iters, seed)


def fcc_periodic(seed: int = 2, ncell: int = 16, p: int = 6, L: float = 30.0,
                 n_fcc: int = 4, n_want: int = 1000, degree: int = 40,
                 iters: int = 20, block: int = 200) -> System:
    """Periodic box with wells on jittered FCC sites (n_fcc^3 conventional cells)."""
    a = L / n_fcc
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    sites = []
    for k in range(n_fcc):
        for j in range(n_fcc):
            for i in range(n_fcc):
                for b in basis:
                    sites.append((np.array([i, j, k]) + b) * a)
    sites = np.array(sites)
    n = len(sites)
    jit = 0.3 * uniform_pm1(seed, STREAM_JITTER, np.arange(3 * n, dtype=np.uint64)).reshape(n, 3)
    centres = np.mod(sites + jit + 0.25 * a, L)
    depths = 1.0 + 2.0 * uniform01(seed, STREAM_DEPTHS, np.arange(n, dtype=np.uint64))
    widths = 0.8 + 0.4 * uniform01(seed, STREAM_WIDTHS, np.arange(n, dtype=np.uint64))
    return System("fcc-periodic-%dc-p%d" % (ncell, p), ncell, p, L, True, centres,
                  depths, widths, n_want, degree, iters, seed, block)


def cubic_sites_nonlocal(seed: int = 3, ncell: int = 20, p: int = 7, L: float = 40.0,
                         n_side: int = 10, n_want: int = 3000, degree: int = 50,
                         iters: int = 10, block: int = 0) -> System:
    """Periodic box, one site per simple-cubic cell: a well plus 4 projectors.

    Projector couplings h are drawn uniform in [0.5, 2] Ha (positive).
    """
    s = L / n_side
    g = (np.arange(n_side) + 0.5) * s
    sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)[:, ::-1].copy()
    n = len(sites)
    jit = 0.3 * uniform_pm1(seed, STREAM_JITTER, np.arange(3 * n, dtype=np.uint64)).reshape(n, 3)
    centres = np.mod(sites + jit, L)
    depths = 1.0 + 2.0 * uniform01(seed, STREAM_DEPTHS, np.arange(n, dtype=np.uint64))
    widths = 0.8 + 0.4 * uniform01(seed, STREAM_WIDTHS, np.arange(n, dtype=np.uint64))
    h = 0.5 + 1.5 * uniform01(seed, STREAM_NL_H, np.arange(4 * n, dtype=np.uint64)).reshape(n, 4)
    return System("nonlocal-periodic-%dc-p%d" % (ncell, p), ncell, p, L, True, centres,
                  depths, widths, n_want, degree, iters, seed, block,
                  nl_centres=centres.copy(), nl_h=h)


def batched_systems(seed: int = 4, count: int = 64, p: int = 5, h: float = 1.5,
                    degree: int = 30, iters: int = 6):
    """Uneven non-periodic systems: n ~ U{4..12} cells per side, 2-64 wells
    in the inner 80 % of the box, N log-uniform in [16, 400] capped at M/8."""
    out = []
    u = uniform01(seed, STREAM_SYSTEMS, np.arange(3 * count, dtype=np.uint64)).reshape(count, 3)
    for s in range(count):
        n = 4 + int(u[s, 0] * 9)
        L = n * h
        nw = 2 + int(u[s, 1] * 63)
        M = (n * p - 1) ** 3
        nwant = int(round(math.exp(math.log(16) + u[s, 2] * (math.log(400) - math.log(16)))))
        nwant = max(8, min(nwant, M // 8))
        c, d, w = _wells_uniform(seed * 1000 + s, nw, np.full(3, 0.1 * L), np.full(3, 0.9 * L))
        out.append(System("batch-%d" % s, n, p, L, False, c, d, w, nwant, degree, iters,
                          seed * 1000 + s))
    return out


def perturbed_depths(sys: System, seed: int, step: int, rel: float = 0.01) -> np.ndarray:
    """Well depths scaled by (1 + rel * xi), xi ~ U(-sqrt3, sqrt3) (unit variance)."""
    xi = math.sqrt(3.0) * uniform_pm1(seed, STREAM_NOISE,
                                      np.arange(len(sys.depths), dtype=np.uint64)
                                      + np.uint64(step) * np.uint64(1 << 20))
    return sys.depths * (1.0 + rel * xi)


STREAM_ARRIVALS = 10


def serving_requests(seed: int = 5, count: int = 24, dof_range=(2.0e4, 2.0e6),
                     n_range=(32, 1000), h: float = 2.0, well_volume: float = 125.0,
                     degree: int = 30, iters: int = 24, resolves: int = 5):
    """Stream of eigensolve requests for the serving loop.

    Per request: DOFs log-uniform in dof_range, p ~ U{5,6,7}, n = round(DOF^(1/3) / p)
    cells per side (at least 2) of size h (periodic), one well per
    ``well_volume`` bohr^3 at uniform centres, N log-uniform in n_range
    (capped at M/8), and ``resolves`` follow-up well-depth sets from
    ``perturbed_depths`` (1 % noise, step k = 1..resolves).  Returns a list of
    (System, [depths of re-solve 1..resolves]).
    """
    u = uniform01(seed, STREAM_SYSTEMS, np.arange(3 * count, dtype=np.uint64)).reshape(count, 3)
    out = []
    for s in range(count):
        dof = math.exp(math.log(dof_range[0]) + u[s, 0] * (math.log(dof_range[1]) - math.log(dof_range[0])))
        p = 5 + min(2, int(u[s, 1] * 3))
        n = max(2, int(round(dof ** (1.0 / 3.0) / p)))
        L = n * h
        nw = max(1, int(round(L ** 3 / well_volume)))
        M = (n * p) ** 3
        nwant = math.exp(math.log(n_range[0]) + u[s, 2] * (math.log(n_range[1]) - math.log(n_range[0])))
        nwant = max(8, min(int(round(nwant)), M // 8))
        sseed = seed * 1000 + s
        c, d, w = _wells_uniform(sseed, nw, np.zeros(3), np.full(3, L))
        sys = System("serve-%d" % s, n, p, L, True, c, d, w, nwant, degree, iters, sseed)
        seq = [perturbed_depths(sys, sseed, k) for k in range(1, resolves + 1)]
        out.append((sys, seq))
    return out


def poisson_arrivals(seed: int, count: int, rate: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate (exponential gaps)."""
    u = uniform01(seed, STREAM_ARRIVALS, np.arange(count, dtype=np.uint64))
    return np.cumsum(-np.log1p(-u) / rate)
