"""ctypes binding of libchfsi (include/chfsi.h): argument marshalling only.

Every method of :class:`Context` calls the C entry point of the same name
(``chfsi_<name>``); all arithmetic runs in the library's CUDA kernels.  Device
buffers are passed as torch CUDA tensors (their ``data_ptr``), host arrays as
numpy arrays.  There is no CPU fallback: loading fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchfsi.so")

FP64, MIXED_TF32X3, MIXED_TF32, MIXED_BF16X3, MIXED_F16X2 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": FP64, "mixed": MIXED_TF32X3, "tf32x3": MIXED_TF32X3, "tf32": MIXED_TF32,
              "bf16x3": MIXED_BF16X3, "f16x2": MIXED_F16X2}

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_NOT_SPD", 5: "ERR_EIG",
          6: "ERR_STATE", 7: "ERR_TIMEOUT"}


class ChfsiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class MeshDesc(C.Structure):
    _fields_ = [("ncell", C.c_int * 3), ("len", C.c_double * 3), ("p", C.c_int),
                ("periodic", C.c_int * 3), ("quad_points", C.c_int)]


def _axes(periodic):
    """Per-axis periodic flags (x, y, z) from one flag or three."""
    if np.ndim(periodic) == 0:
        return (int(bool(periodic)),) * 3
    t = tuple(int(bool(v)) for v in periodic)
    if len(t) != 3:
        raise ValueError("periodic: one flag or three (x, y, z)")
    return t


MAX_SOLVES = 16


class PartitionInfo(C.Structure):
    _fields_ = [("ncells", C.c_int64), ("nlocal", C.c_int64), ("nhalo", C.c_int64),
                ("nneighbors", C.c_int), ("grid", C.c_int * 3)]


class ScfParams(C.Structure):
    _fields_ = [("nnuclei", C.c_int), ("xyz", C.POINTER(C.c_double)), ("Z", C.POINTER(C.c_double)),
                ("sigma", C.POINTER(C.c_double)), ("n_states", C.c_int), ("kT", C.c_double),
                ("degree", C.c_int), ("passes", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int),
                ("beta", C.c_double), ("depth", C.c_int), ("seed", C.c_uint64),
                ("poisson_tol", C.c_double), ("lanczos_steps", C.c_int)]


class Request(C.Structure):
    _fields_ = [("mesh", MeshDesc), ("n", C.c_int), ("nwells", C.c_int),
                ("xyz", C.POINTER(C.c_double)), ("depth", C.POINTER(C.c_double)),
                ("width", C.POINTER(C.c_double)), ("resolves", C.c_int),
                ("depth_seq", C.POINTER(C.c_double)), ("degree", C.c_int), ("iters", C.c_int),
                ("warm_iters", C.c_int), ("tol", C.c_double), ("n_check", C.c_int),
                ("prec", C.c_int), ("seed", C.c_uint64), ("polish_iters", C.c_int),
                ("polish_degree", C.c_int)]


class Result(C.Structure):
    _fields_ = [("done", C.c_int), ("status", C.c_int), ("nsolves", C.c_int),
                ("queue_ms", C.c_double), ("first_ms", C.c_double),
                ("total_ms", C.c_double), ("est_bytes", C.c_size_t), ("used_bytes", C.c_size_t),
                ("solve_ms", C.c_double * MAX_SOLVES), ("max_residual", C.c_double * MAX_SOLVES),
                ("max_gresidual", C.c_double * MAX_SOLVES), ("iters", C.c_int * MAX_SOLVES),
                ("error", C.c_char * 160)]


_lib = None
_dp = C.POINTER(C.c_double)
_vp = C.c_void_p
_i64 = C.c_int64

_SIGS = {
    "chfsi_create": (C.c_int, [C.POINTER(MeshDesc), _vp, C.POINTER(_vp)]),
    "chfsi_destroy": (C.c_int, [_vp]),
    "chfsi_last_error": (C.c_char_p, [_vp]),
    "chfsi_num_dofs": (_i64, [_vp]),
    "chfsi_device_bytes": (_i64, [_vp]),
    "chfsi_mass_diag": (C.c_int, [_vp, _dp]),
    "chfsi_set_potential_gaussians": (C.c_int, [_vp, C.c_int, _dp, _dp, _dp]),
    "chfsi_set_potential_qp": (C.c_int, [_vp, _dp, _i64]),
    "chfsi_set_projectors": (C.c_int, [_vp, C.c_int, _dp, _dp, C.c_double, C.c_double]),
    "chfsi_build": (C.c_int, [_vp]),
    "chfsi_set_blocking": (C.c_int, [_vp, C.c_int, C.c_int]),
    "chfsi_set_cell_tile": (C.c_int, [_vp, C.c_int]),
    "chfsi_set_gemm_kernels": (C.c_int, [_vp, C.c_int, C.c_int]),
    "chfsi_set_filter_lanes": (C.c_int, [_vp, C.c_int]),
    "chfsi_apply_kpoint_mixed": (C.c_int, [_vp, _vp, C.c_int64, _vp, C.c_int64, C.c_int]),
    "chfsi_solve_kpoint_prec": (C.c_int, [_vp, _vp, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                                          _vp]),
    "chfsi_autotune": (C.c_int, [_vp, _vp, _i64, C.c_int, C.c_int, C.POINTER(C.c_int),
                                 C.POINTER(C.c_int), _dp]),
    "chfsi_fill_uniform": (C.c_int, [_vp, _vp, _i64, _i64, C.c_int, C.c_uint64, C.c_uint64, C.c_int]),
    "chfsi_apply": (C.c_int, [_vp, _vp, _i64, _vp, _i64, C.c_int, C.c_int]),
    "chfsi_apply_noalloc": (C.c_int, [_vp, _vp, _i64, _vp, _i64, C.c_int]),
    "chfsi_filter": (C.c_int, [_vp, _vp, _i64, C.c_int, C.c_int, C.c_double, C.c_double,
                               C.c_double, C.c_int]),
    "chfsi_cholgs": (C.c_int, [_vp, _vp, _i64, C.c_int, C.c_int]),
    "chfsi_rayleigh_ritz": (C.c_int, [_vp, _vp, _i64, C.c_int, C.c_int, _dp]),
    "chfsi_residuals": (C.c_int, [_vp, _vp, _i64, C.c_int, C.c_int, _dp, _dp, _dp]),
    "chfsi_bounds": (C.c_int, [_vp, C.c_int, C.c_uint64, _dp]),
    "chfsi_solve": (C.c_int, [_vp, _vp, _i64, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                              C.c_int, C.c_int, _dp, C.POINTER(C.c_int)]),
    "chfsi_solve_polish": (C.c_int, [_vp, _vp, _i64, C.c_int, C.c_int, C.c_int, C.c_double,
                                     C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _i64,
                                     _dp, C.POINTER(C.c_int)]),
    "chfsi_step_host": (C.c_int, [_vp, _vp, _i64, _vp, _i64, C.c_int, C.c_int, C.c_double,
                                  C.c_double, C.c_double, C.c_int, C.c_int, _dp, _dp]),
    "chfsi_unscale": (C.c_int, [_vp, _vp, _i64, C.c_int, C.c_int]),
    "chfsi_rayleigh_ritz_split": (C.c_int, [_vp, _vp, _i64, C.c_int, C.c_int, _vp, _i64, C.c_int, _dp]),
    "chfsi_fermi_level": (C.c_int, [C.c_int, _dp, C.c_int, C.c_double, C.c_double, _dp, _dp]),
    "chfsi_density": (C.c_int, [_vp, _vp, _i64, C.c_int, _vp, _i64, C.c_int, _dp, C.c_int, _vp]),
    "chfsi_last_timings": (C.c_int, [_vp, _dp]),
    "chfsi_kernel_launches": (_i64, []),
    "chfsi_batch_create": (C.c_int, [C.c_int, C.POINTER(_vp), _vp, C.POINTER(_vp)]),
    "chfsi_batch_destroy": (C.c_int, [_vp]),
    "chfsi_batch_last_error": (C.c_char_p, [_vp]),
    "chfsi_batch_filter": (C.c_int, [_vp, C.POINTER(_vp), C.POINTER(_i64), C.POINTER(C.c_int), C.c_int,
                                     _dp, _dp, _dp, C.c_int]),
    "chfsi_batch_autotune": (C.c_int, [_vp, C.POINTER(_vp), C.POINTER(_i64), C.POINTER(C.c_int),
                                       C.c_int, C.POINTER(C.c_int), _dp]),
    "chfsi_batch_candidates": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int]),
    "chfsi_batch_set_candidate": (C.c_int, [_vp, C.c_int]),
    "chfsi_batch_solve": (C.c_int, [_vp, C.POINTER(_vp), C.POINTER(_i64), C.POINTER(C.c_int), C.c_int,
                                    C.c_int, _dp, C.c_int, C.c_int, C.POINTER(_dp)]),
    "chfsi_server_create": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(_vp)]),
    "chfsi_server_submit": (C.c_int, [_vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "chfsi_server_poll": (C.c_int, [_vp, C.c_uint64, C.c_int, C.POINTER(Result), _dp]),
    "chfsi_server_estimate": (C.c_size_t, [C.POINTER(Request)]),
    "chfsi_server_destroy": (C.c_int, [_vp]),
    "chfsi_set_kernel_timing": (C.c_int, [_vp, C.c_int]),
    "chfsi_set_kpoint": (C.c_int, [_vp, _dp]),
    "chfsi_apply_kpoint": (C.c_int, [_vp, _vp, _i64, _vp, _i64, C.c_int]),
    "chfsi_bounds_kpoint": (C.c_int, [_vp, C.c_int, C.c_uint64, _dp]),
    "chfsi_solve_kpoint": (C.c_int, [_vp, _vp, _i64, C.c_int, C.c_int, C.c_int, C.c_double, _dp]),
    "chfsi_set_potential_qp_device": (C.c_int, [_vp, _vp]),
    "chfsi_poisson": (C.c_int, [_vp, _vp, _vp, C.c_double, C.c_int, C.POINTER(C.c_int), _dp]),
    "chfsi_scf": (C.c_int, [_vp, C.POINTER(ScfParams), _vp, _i64, _dp, _dp, _dp, _dp, _dp,
                            C.POINTER(C.c_int)]),
    "chfsi_set_fp64_operator": (C.c_int, [_vp, C.c_int]),
    "chfsi_set_cell_gather": (C.c_int, [_vp, C.c_int]),
    "chfsi_fp64_operator": (C.c_int, [_vp]),
    "chfsi_debug_withhold_arrival": (C.c_int, [_vp, C.c_int]),
    "chfsi_partition_sizes": (C.c_int, [C.POINTER(MeshDesc), C.c_int, C.c_int,
                                        C.POINTER(PartitionInfo)]),
    "chfsi_partition_fill": (C.c_int, [C.POINTER(MeshDesc), C.c_int, C.c_int, _vp, _vp, _vp, _vp,
                                       _vp, _vp]),
    "chfsi_kernel_timings": (C.c_int, [_vp, _dp]),
}


def load(path: str | None = None):
    """Load libchfsi.so (raises if it is missing: there is no fallback)."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libchfsi.so not built at %s: run __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


def kernel_launches() -> int:
    """Kernels launched by libchfsi so far (chfsi_kernel_launches)."""
    return int(load().chfsi_kernel_launches())


def exported_symbols():
    return list(_SIGS)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _host(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _prec(p):
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _dev(t, prec=None):
    """(pointer, leading dimension, ncol) of a 2-D row-major CUDA tensor."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("device buffers must be CUDA tensors")
    if t.dim() == 1:
        return t.data_ptr(), 1, 1
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a 2-D tensor with unit column stride")
    if prec is not None:
        want = torch.float64 if prec == FP64 else torch.float32
        if t.dtype != want:
            raise TypeError("precision %d needs dtype %s, got %s" % (prec, want, t.dtype))
    return t.data_ptr(), t.stride(0), t.shape[1]


class Context:
    """One discretised problem on the current CUDA device (chfsi_ctx)."""

    def __init__(self, ncell, length, p, periodic=True, quad_points=0, stream=None):
        """``periodic``: one flag for all axes or three (x, y, z); a Dirichlet
        axis drops the nodes of its two faces."""
        lib = load()
        if np.isscalar(ncell):
            ncell = (ncell,) * 3
        if np.isscalar(length):
            length = (float(length),) * 3
        d = MeshDesc((C.c_int * 3)(*ncell), (C.c_double * 3)(*length), int(p),
                     (C.c_int * 3)(*_axes(periodic)), int(quad_points))
        h = _vp()
        s = _vp(stream.cuda_stream) if stream is not None else _vp(None)
        self._lib = lib
        st = lib.chfsi_create(C.byref(d), s, C.byref(h))
        if st != 0:
            raise ChfsiError(st, "chfsi_create failed")
        self._h = h
        self.ndofs = lib.chfsi_num_dofs(h)
        self._ncells = int(ncell[0]) * int(ncell[1]) * int(ncell[2])
        self._q = int(quad_points) if quad_points else int(p) + 2

    def _check(self, st):
        if st != 0:
            raise ChfsiError(st, self._lib.chfsi_last_error(self._h).decode())

    def destroy(self):
        if getattr(self, "_h", None):
            self._lib.chfsi_destroy(self._h)
            self._h = None

    close = destroy

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def last_error(self) -> str:
        return self._lib.chfsi_last_error(self._h).decode()

    def device_bytes(self) -> int:
        return self._lib.chfsi_device_bytes(self._h)

    def mass_diag(self) -> np.ndarray:
        out = np.empty(self.ndofs)
        self._check(self._lib.chfsi_mass_diag(self._h, _ptr(out)))
        return out

    def set_potential_gaussians(self, centres, depths, widths):
        n = len(depths)
        c, d, w = _host(centres, 3 * n), _host(depths, n), _host(widths, n)
        self._check(self._lib.chfsi_set_potential_gaussians(self._h, n, _ptr(c), _ptr(d), _ptr(w)))

    def set_potential_qp(self, values=None):
        """General V_eff at the Gauss points (chfsi_set_potential_qp): ncells * q^3
        values, cells x fastest, point a + q (b + q c); added to the wells.
        None clears."""
        if values is None:
            self._check(self._lib.chfsi_set_potential_qp(self._h, None, 0))
            return
        v = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(-1))
        self._check(self._lib.chfsi_set_potential_qp(self._h, _ptr(v), int(v.size)))

    def set_projectors(self, centres, h, sigma=0.8, rcut=3.0):
        n = len(centres)
        c, hh = _host(centres, 3 * n), _host(h, 4 * n)
        self._check(self._lib.chfsi_set_projectors(self._h, n, _ptr(c), _ptr(hh), sigma, rcut))

    def build(self):
        self._check(self._lib.chfsi_build(self._h))

    def set_blocking(self, filter_block=200, diag_block=1):
        self._check(self._lib.chfsi_set_blocking(self._h, int(filter_block), int(diag_block)))

    def set_cell_tile(self, tile=64):
        self._check(self._lib.chfsi_set_cell_tile(self._h, int(tile)))

    def set_filter_lanes(self, lanes=1):
        """Column groups filtered concurrently on their own streams (mixed precisions)."""
        self._check(self._lib.chfsi_set_filter_lanes(self._h, int(lanes)))

    def set_gemm_kernels(self, tall=-1, gram=-1):
        """Tile kernels of the mixed block products: -1 by size, 0 = 128 x 128, 1 = 256-row."""
        self._check(self._lib.chfsi_set_gemm_kernels(self._h, int(tall), int(gram)))

    def autotune(self, X, prec="mixed"):
        """(block, tile, {(block, tile): ms}) chosen by chfsi_autotune."""
        pr = _prec(prec)
        p, ld, n = _dev(X, pr)
        ms = np.zeros(6)
        blk, tile = C.c_int(0), C.c_int(0)
        self._check(self._lib.chfsi_autotune(self._h, p, ld, n, pr, C.byref(blk), C.byref(tile),
                                             _ptr(ms)))
        blocks = []
        for bk in (200, (n + 1) // 2, n):
            bk = max(1, min(bk, n))
            if bk not in blocks:
                blocks.append(bk)
        tiles = (64, 128) if pr != FP64 else (64,)
        cands = [(bk, t) for bk in blocks for t in tiles]
        return blk.value, tile.value, {c: float(ms[i]) for i, c in enumerate(cands)}

    def fill_uniform(self, X, seed, stream=1, prec="fp64"):
        pr = _prec(prec)
        ptr, ld, ncol = _dev(X, pr)
        self._check(self._lib.chfsi_fill_uniform(self._h, ptr, ld, X.shape[0], ncol, seed, stream, pr))

    def apply(self, X, Y, prec="fp64"):
        pr = _prec(prec)
        px, ldx, n = _dev(X, pr)
        py, ldy, _ = _dev(Y, pr)
        self._check(self._lib.chfsi_apply(self._h, px, ldx, py, ldy, n, pr))

    def apply_noalloc(self, X, Y):
        """Y = H~ X in binary64 through chfsi_apply_noalloc (no device allocation:
        the assembly scratch is the library's fixed 64 MiB device array)."""
        px, ldx, n = _dev(X, FP64)
        py, ldy, _ = _dev(Y, FP64)
        self._check(self._lib.chfsi_apply_noalloc(self._h, px, ldx, py, ldy, n))

    def set_potential_qp_device(self, v):
        """V_eff at the Gauss points from a CUDA float64 tensor (ncells * q^3)."""
        import torch
        if not isinstance(v, torch.Tensor) or not v.is_cuda or v.dtype != torch.float64 \
                or not v.is_contiguous():
            raise TypeError("v: contiguous CUDA float64 tensor")
        self._check(self._lib.chfsi_set_potential_qp_device(self._h, _vp(v.data_ptr())))

    def poisson(self, f, phi, tol=1e-12, max_iter=20000):
        """phi (CUDA float64, M) of -(1/4 pi) lap phi = f (CUDA float64 at the Gauss
        points); returns (CG iterations, relative residual)."""
        it, rel = C.c_int(0), np.zeros(1)
        self._check(self._lib.chfsi_poisson(self._h, _vp(f.data_ptr()), _vp(phi.data_ptr()),
                                            float(tol), int(max_iter), C.byref(it), _ptr(rel)))
        return it.value, float(rel[0])

    def scf(self, X, centres, Z, sigma, kT=0.01, degree=20, passes=2, tol=1e-9, max_iter=60,
            beta=0.5, depth=6, seed=1, poisson_tol=1e-13, lanczos_steps=20):
        """Algorithm scf on a periodic Gaussian-charge system (chfsi_scf); X is a
        CUDA float64 (M x n_states) work block.  Returns a dict with rho (Gauss
        points), evals, occ, mu, residuals."""
        px, ldx, n = _dev(X, FP64)
        xyz = _host(centres).reshape(-1)
        z, sg = _host(Z), _host(sigma)
        prm = ScfParams(int(z.size), _ptr(xyz), _ptr(z), _ptr(sg), int(n), float(kT), int(degree),
                        int(passes), float(tol), int(max_iter), float(beta), int(depth), int(seed),
                        float(poisson_tol), int(lanczos_steps))
        q = self._q
        rho = np.empty(self._ncells * q ** 3)
        ev, occ, mu = np.empty(n), np.empty(n), np.zeros(1)
        hist = np.zeros(max_iter)
        it = C.c_int(0)
        self._check(self._lib.chfsi_scf(self._h, C.byref(prm), px, ldx, _ptr(rho), _ptr(ev), _ptr(occ),
                                        _ptr(mu), _ptr(hist), C.byref(it)))
        return {"rho": rho, "evals": ev, "occ": occ, "mu": float(mu[0]),
                "residuals": hist[:it.value].copy(), "iters": it.value}

    # ------------------------------------------------------------ k-points
    @staticmethod
    def _cdev(t):
        """(pointer, ld in doubles, n complex vectors) of a CUDA complex128 tensor (M x n)."""
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.complex128 \
                or t.dim() != 2 or t.stride(1) != 1:
            raise TypeError("k-point blocks: 2-D CUDA complex128 tensors with unit column stride")
        return t.data_ptr(), 2 * t.stride(0), t.shape[1]

    def set_kpoint(self, k):
        kk = _host(k, 3)
        self._check(self._lib.chfsi_set_kpoint(self._h, _ptr(kk)))

    def apply_kpoint(self, X, Y):
        px, ldx, n = self._cdev(X)
        py, ldy, n2 = self._cdev(Y)
        if n2 != n:
            raise ValueError("X and Y need the same number of columns")
        self._check(self._lib.chfsi_apply_kpoint(self._h, px, ldx, py, ldy, n))

    def bounds_kpoint(self, steps=20, seed=1) -> float:
        b = np.zeros(1)
        self._check(self._lib.chfsi_bounds_kpoint(self._h, int(steps), int(seed), _ptr(b)))
        return float(b[0])

    def solve_kpoint(self, X, iters, degree, b, prec="fp64"):
        """ChFSI at k on a complex128 block; prec "bf16x3" filters in mixed precision."""
        px, ldx, n = self._cdev(X)
        ev = np.empty(n)
        self._check(self._lib.chfsi_solve_kpoint_prec(self._h, px, ldx, n, int(iters), int(degree), float(b),
                                                      _prec(prec), _ptr(ev)))
        return ev

    def apply_kpoint_mixed(self, X, Y):
        """Y = H~(k) X on complex64 blocks (BF16x3 cell products)."""
        import torch
        for t in (X, Y):
            if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.complex64 \
                    or t.dim() != 2 or t.stride(1) != 1:
                raise TypeError("mixed k-point blocks: 2-D CUDA complex64 tensors with unit column stride")
        if X.shape != Y.shape:
            raise ValueError("X and Y need the same shape")
        self._check(self._lib.chfsi_apply_kpoint_mixed(self._h, X.data_ptr(), 2 * X.stride(0), Y.data_ptr(),
                                                       2 * Y.stride(0), X.shape[1]))

    def set_cell_gather(self, mode):
        """BF16x3 cell kernel: "registers" (register gather, one ring), "async"
        (rows staged by bulk copies) or "rings" (register gather, separate matrix
        and Y rings)."""
        self._check(self._lib.chfsi_set_cell_gather(self._h, {"registers": 0, "async": 1, "rings": 2, "rings4": 3, "whole": 4, "tiles": 5, "tiles2": 6}[mode]))

    def set_fp64_operator(self, op):
        """Binary64 cell operator: "cells" (stored cell matrices), "matrix-free"
        (sum factorisation) or "default" (chfsi_set_fp64_operator)."""
        code = {"default": -1, "cells": 0, "matrix-free": 1}[op]
        self._check(self._lib.chfsi_set_fp64_operator(self._h, code))

    @property
    def fp64_operator(self):
        return ("cells", "matrix-free")[self._lib.chfsi_fp64_operator(self._h)]

    def debug_withhold_arrival(self, on):
        """Test hook of the bounded device waits (chfsi_debug_withhold_arrival)."""
        self._check(self._lib.chfsi_debug_withhold_arrival(self._h, int(bool(on))))

    def filter(self, X, degree, a, b, a0, prec="fp64"):
        pr = _prec(prec)
        px, ldx, n = _dev(X, pr)
        self._check(self._lib.chfsi_filter(self._h, px, ldx, n, degree, a, b, a0, pr))

    def cholgs(self, X, prec="fp64"):
        pr = _prec(prec)
        px, ldx, n = _dev(X, pr)
        self._check(self._lib.chfsi_cholgs(self._h, px, ldx, n, pr))

    def rayleigh_ritz(self, X, prec="fp64") -> np.ndarray:
        pr = _prec(prec)
        px, ldx, n = _dev(X, pr)
        ev = np.empty(n)
        self._check(self._lib.chfsi_rayleigh_ritz(self._h, px, ldx, n, pr, _ptr(ev)))
        return ev

    def residuals(self, X, evals, prec="fp64"):
        pr = _prec(prec)
        px, ldx, n = _dev(X, pr)
        ev = _host(evals, n)
        r, g = np.empty(n), np.empty(n)
        self._check(self._lib.chfsi_residuals(self._h, px, ldx, n, pr, _ptr(ev), _ptr(r), _ptr(g)))
        return r, g

    def bounds(self, steps=20, seed=1) -> float:
        b = np.zeros(1)
        self._check(self._lib.chfsi_bounds(self._h, int(steps), int(seed), _ptr(b)))
        return float(b[0])

    def solve(self, X, iters, degree, b, tol=0.0, n_check=0, prec="fp64"):
        pr = _prec(prec)
        px, ldx, n = _dev(X, pr)
        ev = np.empty(n)
        done = C.c_int(0)
        self._check(self._lib.chfsi_solve(self._h, px, ldx, n, int(iters), int(degree), float(b),
                                          float(tol), int(n_check), pr, _ptr(ev), C.byref(done)))
        return ev, done.value

    def solve_polish(self, X, iters, degree, b, polish_iters=1, polish_degree=None, X64=None,
                     tol=0.0, n_check=0, prec="bf16x3"):
        """Mixed-precision solve on the binary32 block X, then ``polish_iters``
        binary64 iterations (degree ``polish_degree``, default ``degree``) on a
        binary64 copy (``X64`` when given, a CUDA float64 tensor of X's shape);
        X receives the polished block rounded to binary32."""
        pr = _prec(prec)
        px, ldx, n = _dev(X, pr)
        p64, ld64 = None, 0
        if X64 is not None:
            p64, ld64, n64 = _dev(X64, FP64)
            if n64 != n:
                raise ValueError("X64 needs %d columns" % n)
        ev = np.empty(n)
        done = C.c_int(0)
        self._check(self._lib.chfsi_solve_polish(
            self._h, px, ldx, n, int(iters), int(degree), float(b), float(tol), int(n_check), pr,
            int(polish_iters), int(polish_degree or degree), p64, ld64, _ptr(ev), C.byref(done)))
        return ev, done.value

    def step_host(self, X_host, X, degree, a, b, a0, prec="bf16x3", copy_mode=0):
        """One ChFSI iteration on a block in host memory (chfsi_step_host):
        ``X_host`` a CPU tensor (pinned for the fast path), ``X`` a CUDA tensor
        of the same shape used as the device copy.  Returns (Ritz values,
        [h2d_ms, step_ms, d2h_ms])."""
        import torch
        pr = _prec(prec)
        px, ldx, n = _dev(X, pr)
        if not isinstance(X_host, torch.Tensor) or X_host.is_cuda or X_host.dim() != 2 \
                or X_host.stride(1) != 1 or X_host.dtype != X.dtype or X_host.shape != X.shape:
            raise ValueError("X_host: a CPU tensor with X's shape, dtype and unit column stride")
        ev, ms = np.empty(n), np.zeros(3)
        self._check(self._lib.chfsi_step_host(self._h, _vp(X_host.data_ptr()), X_host.stride(0), px,
                                              ldx, n, int(degree), float(a), float(b), float(a0),
                                              pr, int(copy_mode), _ptr(ev), _ptr(ms)))
        return ev, ms

    def rayleigh_ritz_split(self, X, Xfr, prec="fp64") -> np.ndarray:
        """Algorithm rr: the n_fr = Xfr.shape[1] largest Ritz pairs; Xfr <- X Q_fr."""
        pr = _prec(prec)
        px, ldx, n = _dev(X, pr)
        pf, ldf, nfr = _dev(Xfr, pr)
        ev = np.empty(nfr)
        self._check(self._lib.chfsi_rayleigh_ritz_split(self._h, px, ldx, n, nfr, pf, ldf, pr,
                                                        _ptr(ev)))
        return ev

    def density(self, X, rho, Xfr=None, occ_fr=None, prec="fp64"):
        """Algorithm dc: rho (device float64, ncells * q^3) at the Gauss points."""
        import torch
        pr = _prec(prec)
        px, ldx, n = _dev(X, pr)
        if not (isinstance(rho, torch.Tensor) and rho.is_cuda and rho.dtype == torch.float64):
            raise TypeError("rho must be a float64 CUDA tensor")
        if Xfr is not None and Xfr.shape[1] > 0:
            pf, ldf, nfr = _dev(Xfr, pr)
            occ = _host(occ_fr, nfr)
        else:
            pf, ldf, nfr, occ = None, 1, 0, np.zeros(1)
        self._check(self._lib.chfsi_density(self._h, px, ldx, n, pf, ldf, nfr, _ptr(occ), pr,
                                            rho.data_ptr()))

    def unscale(self, X, prec="fp64"):
        pr = _prec(prec)
        px, ldx, n = _dev(X, pr)
        self._check(self._lib.chfsi_unscale(self._h, px, ldx, n, pr))

    def set_kernel_timing(self, on=True):
        self._check(self._lib.chfsi_set_kernel_timing(self._h, int(bool(on))))

    def kernel_timings(self) -> np.ndarray:
        """[cell-product ms, assembly ms, cell launches, assembly launches, projector ms,
        projector launch pairs] since the last call."""
        out = np.zeros(6)
        self._check(self._lib.chfsi_kernel_timings(self._h, _ptr(out)))
        return out

    def last_timings(self) -> np.ndarray:
        out = np.zeros(4)
        self._check(self._lib.chfsi_last_timings(self._h, _ptr(out)))
        return out


class Batch:
    """Batched filtering / ChFSI of several built Contexts (chfsi_batch_*)."""

    def __init__(self, contexts, stream=None):
        lib = load()
        self._lib = lib
        self.contexts = list(contexts)
        arr = (_vp * len(self.contexts))(*[c._h for c in self.contexts])
        h = _vp()
        s = _vp(stream.cuda_stream) if stream is not None else _vp(None)
        st = lib.chfsi_batch_create(len(self.contexts), arr, s, C.byref(h))
        if st != 0:
            raise ChfsiError(st, "chfsi_batch_create failed")
        self._h = h

    def _check(self, st):
        if st != 0:
            raise ChfsiError(st, self._lib.chfsi_batch_last_error(self._h).decode())

    def destroy(self):
        if getattr(self, "_h", None):
            self._lib.chfsi_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    @staticmethod
    def _blocks(X, prec):
        ptrs, lds, ncols = [], [], []
        for x in X:
            p, ld, n = _dev(x, prec)
            ptrs.append(p)
            lds.append(ld)
            ncols.append(n)
        k = len(X)
        return (_vp * k)(*ptrs), (_i64 * k)(*lds), (C.c_int * k)(*ncols)

    def filter(self, X, degree, a, b, a0, prec="mixed"):
        pr = _prec(prec)
        p, ld, n = self._blocks(X, pr)
        a, b, a0 = _host(a), _host(b), _host(a0)
        self._check(self._lib.chfsi_batch_filter(self._h, p, ld, n, int(degree), _ptr(a), _ptr(b),
                                                 _ptr(a0), pr))

    def candidates(self):
        k = self._lib.chfsi_batch_candidates(self._h, None, None, 0)
        bn, st = (C.c_int * k)(), (C.c_int * k)()
        self._lib.chfsi_batch_candidates(self._h, bn, st, k)
        return list(zip(list(bn), list(st)))

    def set_candidate(self, k):
        self._check(self._lib.chfsi_batch_set_candidate(self._h, int(k)))

    def autotune(self, X, prec="mixed"):
        pr = _prec(prec)
        p, ld, n = self._blocks(X, pr)
        k = len(self.candidates())
        ms = np.zeros(k)
        choice = C.c_int(-1)
        self._check(self._lib.chfsi_batch_autotune(self._h, p, ld, n, pr, C.byref(choice), _ptr(ms)))
        return choice.value, ms

    def solve(self, X, iters, degree, bounds, filter_prec="mixed", orth_prec="fp64"):
        p, ld, n = self._blocks(X, FP64)
        bnd = _host(bounds)
        evs = [np.empty(x.shape[1]) for x in X]
        earr = (_dp * len(X))(*[_ptr(e) for e in evs])
        self._check(self._lib.chfsi_batch_solve(self._h, p, ld, n, int(iters), int(degree), _ptr(bnd),
                                                _prec(filter_prec), _prec(orth_prec), earr))
        return evs


def _request(mesh, n, centres, depths, widths, depth_seq=(), degree=30, iters=20, warm_iters=4,
             tol=0.0, n_check=0, prec="mixed", seed=1, polish_iters=0, polish_degree=0):
    """ctypes Request plus the numpy arrays it points into (kept alive by the caller)."""
    xyz = _host(centres).reshape(-1)
    dep, wid = _host(depths), _host(widths)
    seq = _host(depth_seq).reshape(-1) if len(depth_seq) else np.zeros(0)
    nw = dep.size
    if xyz.size != 3 * nw or wid.size != nw or seq.size % max(nw, 1):
        raise ValueError("inconsistent well arrays")
    resolves = seq.size // nw if nw else len(depth_seq)
    ncell, length, p, periodic = mesh[:4]
    md = MeshDesc((C.c_int * 3)(*ncell), (C.c_double * 3)(*length), int(p),
                  (C.c_int * 3)(*_axes(periodic)), int(mesh[4]) if len(mesh) > 4 else 0)
    r = Request(md, int(n), nw, _ptr(xyz), _ptr(dep), _ptr(wid), int(resolves),
                _ptr(seq) if seq.size else None, int(degree), int(iters), int(warm_iters),
                float(tol), int(n_check), _prec(prec), int(seed), int(polish_iters),
                int(polish_degree))
    return r, (xyz, dep, wid, seq)


class Server:
    """Continuous-batching eigensolve server (chfsi_server_*).

    ``submit`` takes one system -- ``mesh = (ncell, length, p, periodic)``,
    Gaussian wells -- and the depths of its warm re-solves; ``poll`` returns
    a dict with the Ritz values of every solve, the latencies and residuals.
    """

    def __init__(self, hbm_budget_bytes, max_active=4):
        lib = load()
        self._lib = lib
        h = _vp()
        st = lib.chfsi_server_create(int(hbm_budget_bytes), int(max_active), C.byref(h))
        if st != 0:
            raise ChfsiError(st, "chfsi_server_create failed")
        self._h = h
        self._n = {}

    @staticmethod
    def estimate(mesh, n, prec="mixed", nwells=0):
        r, keep = _request(mesh, n, np.zeros((nwells, 3)), np.zeros(nwells), np.ones(nwells),
                           prec=prec)
        return int(load().chfsi_server_estimate(C.byref(r)))

    def submit(self, mesh, n, centres, depths, widths, depth_seq=(), **kw) -> int:
        r, keep = _request(mesh, n, centres, depths, widths, depth_seq, **kw)
        t = C.c_uint64(0)
        st = self._lib.chfsi_server_submit(self._h, C.byref(r), C.byref(t))
        if st != 0:
            raise ChfsiError(st, "chfsi_server_submit rejected the request")
        self._n[t.value] = (int(n), r.resolves + 1)
        return t.value

    def poll(self, ticket, wait=True):
        n, ns = self._n[ticket]
        res = Result()
        ev = np.zeros(ns * n)
        st = self._lib.chfsi_server_poll(self._h, C.c_uint64(ticket), int(bool(wait)), C.byref(res),
                                         _ptr(ev))
        if st != 0:
            raise ChfsiError(st, "chfsi_server_poll failed")
        if not res.done:
            return None
        k = res.nsolves
        return {"status": res.status, "error": res.error.decode(errors="replace"),
                "evals": ev.reshape(ns, n)[:k], "nsolves": k, "iters": list(res.iters[:k]),
                "queue_ms": res.queue_ms, "first_ms": res.first_ms, "total_ms": res.total_ms,
                "est_bytes": res.est_bytes, "used_bytes": res.used_bytes,
                "solve_ms": list(res.solve_ms[:k]), "max_residual": list(res.max_residual[:k]),
                "max_gresidual": list(res.max_gresidual[:k])}

    def destroy(self):
        if getattr(self, "_h", None):
            self._lib.chfsi_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


def fermi_level(evals, n_oc, n_electrons, kT):
    """Algorithm dc, step 1 (chfsi_fermi_level): (mu, occupations)."""
    ev = _host(evals)
    occ = np.empty(ev.size)
    mu = C.c_double(0.0)
    st = load().chfsi_fermi_level(int(ev.size), _ptr(ev), int(n_oc), float(n_electrons), float(kT),
                                  C.byref(mu), _ptr(occ))
    if st != 0:
        raise ChfsiError(st, "chfsi_fermi_level: the states cannot hold that many electrons")
    return mu.value, occ


def partition(ncell, length, p, periodic, nranks, rank):
    """Domain decomposition of the mesh for one rank (chfsi_partition_sizes /
    chfsi_partition_fill): dict with cells, l2g, owner, neighbors, halo (list
    of local-index arrays, one per neighbor) and the rank grid."""
    lib = load()
    if np.isscalar(ncell):
        ncell = (ncell,) * 3
    if np.isscalar(length):
        length = (float(length),) * 3
    d = MeshDesc((C.c_int * 3)(*ncell), (C.c_double * 3)(*length), int(p),
                 (C.c_int * 3)(*_axes(periodic)), 0)
    info = PartitionInfo()
    st = lib.chfsi_partition_sizes(C.byref(d), int(nranks), int(rank), C.byref(info))
    if st != 0:
        raise ChfsiError(st, "chfsi_partition_sizes: no partition of this mesh over %d ranks" % nranks)
    cells = np.empty(info.ncells, np.int32)
    l2g = np.empty(info.nlocal, np.int32)
    owner = np.empty(info.nlocal, np.int32)
    nbr = np.empty(max(info.nneighbors, 1), np.int32)
    hptr = np.empty(info.nneighbors + 1, np.int64)
    halo = np.empty(max(info.nhalo, 1), np.int32)
    vp = lambda a: a.ctypes.data_as(_vp)  # noqa: E731
    st = lib.chfsi_partition_fill(C.byref(d), int(nranks), int(rank), vp(cells), vp(l2g), vp(owner),
                                  vp(nbr), vp(hptr), vp(halo))
    if st != 0:
        raise ChfsiError(st, "chfsi_partition_fill failed")
    k = info.nneighbors
    return {"cells": cells, "l2g": l2g, "owner": owner, "neighbors": nbr[:k].copy(),
            "halo": [halo[hptr[i]:hptr[i + 1]].copy() for i in range(k)],
            "grid": tuple(info.grid)}
