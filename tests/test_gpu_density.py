"""Spectrum-splitting Rayleigh-Ritz and electron density on the GPU against
the oracle (Sec. 3.5, Algorithms rr and dc, Eq. elecDensSP).

Binary64: Ritz values 1e-10, rotated columns 1e-10 (up to sign), density
1e-12 relative.  Mixed (3xTF32 projection and rotation; density interpolated
in binary32, three passes of <= 9 terms, summed in binary32 over 32 columns and
in binary32 pairs across them): Ritz values
1e-5 relative to the spectrum's scale, density 1e-6 relative."""
import numpy as np
import pytest
import torch

from oracle import chfsi as och
from oracle import density as od
from paper_1903_10959_gb300 import workloads as W

from gpu_util import gpu_context, oracle_problem, rel_fro

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _sys(kind):
    if kind == "periodic":
        return W.small_periodic(seed=31, ncell=3, p=4, L=6.0, n_wells=4, n_want=20)
    if kind == "dirichlet":
        s = W.small_periodic(seed=32, ncell=2, p=6, L=5.0, n_wells=2, n_want=14)
        s.periodic = False
        s.centres = 0.1 * s.L + 0.8 * s.centres
        return s
    s = W.small_periodic(seed=33, ncell=3, p=3, L=7.0, n_wells=4, n_want=16)
    s.nl_centres = s.centres[:2].copy()
    s.nl_h = 0.5 + np.arange(8).reshape(2, 4) / 8.0
    return s


@pytest.fixture(scope="module", params=["periodic", "dirichlet", "nonlocal"])
def case(request):
    s = _sys(request.param)
    prob = oracle_problem(s)
    ctx = gpu_context(s)
    n = s.n_sub
    X0 = och.cholgs(W.start_block(s.seed, prob.ndofs, n))
    yield s, prob, ctx, X0
    ctx.destroy()


def _align(A, B):
    sign = np.sign((A * B).sum(0))
    sign[sign == 0] = 1
    return A * sign


@pytest.mark.parametrize("n_fr", [1, 5])
def test_split_rr_fp64(case, n_fr):
    s, prob, ctx, X0 = case
    d_ref, Xfr_ref = od.rayleigh_ritz_split(prob.apply_Htilde, X0, n_fr)
    X = torch.tensor(X0, device=DEV)
    Xfr = torch.zeros((prob.ndofs, n_fr), dtype=torch.float64, device=DEV)
    d = ctx.rayleigh_ritz_split(X, Xfr, prec="fp64")
    assert np.abs(d - d_ref).max() < 1e-10
    got = Xfr.cpu().numpy()
    assert np.abs(_align(got, Xfr_ref) - Xfr_ref).max() < 1e-10
    assert np.array_equal(X.cpu().numpy(), X0)            # X is not modified


def test_split_rr_mixed(case):
    s, prob, ctx, X0 = case
    n_fr = 4
    x32 = X0.astype(np.float32)
    d_ref, Xfr_ref = od.rayleigh_ritz_split(prob.apply_Htilde, x32.astype(np.float64), n_fr)
    X = torch.tensor(x32, device=DEV)
    Xfr = torch.zeros((prob.ndofs, n_fr), dtype=torch.float32, device=DEV)
    ctx.set_blocking(200, 8)
    d = ctx.rayleigh_ritz_split(X, Xfr, prec="mixed")
    scale = max(1.0, np.abs(d_ref).max())
    assert np.abs(d - d_ref).max() < 1e-5 * scale
    got = Xfr.cpu().numpy().astype(np.float64)
    assert rel_fro(_align(got, Xfr_ref), Xfr_ref) < 1e-4


def test_density_fp64(case):
    s, prob, ctx, X0 = case
    n = X0.shape[1]
    n_fr = 5
    d_fr, Xfr_ref = od.rayleigh_ritz_split(prob.apply_Htilde, X0, n_fr)
    mu, occ = od.fermi_level(d_fr, n - n_fr, 2 * (n - n_fr) + 3.3, kT=0.05)
    rho_ref = od.density(prob, X0, Xfr_ref, occ)
    X = torch.tensor(X0, device=DEV)
    Xfr = torch.tensor(Xfr_ref, device=DEV)
    q = prob.basis.q
    rho = torch.empty(prob.mesh.ncells * q ** 3, dtype=torch.float64, device=DEV)
    ctx.density(X, rho, Xfr, occ, prec="fp64")
    got = rho.cpu().numpy().reshape(prob.mesh.ncells, q ** 3)
    assert rel_fro(got, rho_ref) < 1e-12
    # n_fr = 0: n doubly occupied states
    ctx.density(X, rho, prec="fp64")
    got0 = rho.cpu().numpy().reshape(prob.mesh.ncells, q ** 3)
    assert rel_fro(got0, od.density(prob, X0)) < 1e-12


def test_density_mixed_input(case):
    s, prob, ctx, X0 = case
    x32 = X0.astype(np.float32)
    rho_ref = od.density(prob, x32.astype(np.float64))
    X = torch.tensor(x32, device=DEV)
    q = prob.basis.q
    rho = torch.empty(prob.mesh.ncells * q ** 3, dtype=torch.float64, device=DEV)
    ctx.density(X, rho, prec="mixed")
    got = rho.cpu().numpy().reshape(prob.mesh.ncells, q ** 3)
    assert rel_fro(got, rho_ref) < 1e-6             # binary32 interpolation, binary64 sums


def test_full_pipeline_matches_full_rotation(case):
    """GPU split RR -> library Fermi level -> GPU density equals the oracle's
    density of the fully rotated, occupied states."""
    from paper_1903_10959_gb300 import fermi_level
    s, prob, ctx, X0 = case
    n = X0.shape[1]
    n_fr = 6
    X = torch.tensor(X0, device=DEV)
    Xfr = torch.zeros((prob.ndofs, n_fr), dtype=torch.float64, device=DEV)
    d = ctx.rayleigh_ritz_split(X, Xfr, prec="fp64")
    mu, occ = fermi_level(d, n - n_fr, 2 * (n - n_fr) + 5.0, 0.02)
    q = prob.basis.q
    rho = torch.empty(prob.mesh.ncells * q ** 3, dtype=torch.float64, device=DEV)
    ctx.density(X, rho, Xfr, occ, prec="fp64")
    D, XR = och.rayleigh_ritz(prob.apply_Htilde, X0)
    f = np.concatenate([np.ones(n - n_fr), occ])
    ref = od.density(prob, XR * np.sqrt(f)[None, :])
    got = rho.cpu().numpy().reshape(prob.mesh.ncells, q ** 3)
    assert rel_fro(got, ref) < 1e-10


@pytest.mark.parametrize("p,periodic", [(2, True), (5, False), (7, True), (8, True)])
def test_density_binary32_kernel_degrees(p, periodic):
    """The binary32 density kernel (lane = column, 32-column chunks, sums over
    the columns by a warp reduce-scatter, binary32-pair accumulation across
    chunks) against the oracle at p = 2 ... 8: several chunks with a ragged
    tail for both blocks, partially occupied states with negative weights,
    a Dirichlet mesh; and against the binary64 kernel on the same values."""
    s = W.small_periodic(seed=40 + p, ncell=2, p=p, L=2.0 + 0.4 * p, n_wells=2, n_want=8)
    if not periodic:
        s.periodic = False
        s.centres = 0.1 * s.L + 0.8 * s.centres
    prob = oracle_problem(s)
    ctx = gpu_context(s)
    try:
        n, n_fr = 70, 37
        x32 = W.start_block(s.seed, prob.ndofs, n).astype(np.float32)
        f32 = W.start_block(s.seed + 1, prob.ndofs, n_fr).astype(np.float32)
        occ = np.linspace(0.05, 0.95, n_fr)
        rho_ref = od.density(prob, x32.astype(np.float64), f32.astype(np.float64), occ)
        q = prob.basis.q
        rho = torch.empty(prob.mesh.ncells * q ** 3, dtype=torch.float64, device=DEV)
        ctx.density(torch.tensor(x32, device=DEV), rho, torch.tensor(f32, device=DEV), occ, prec="mixed")
        got = rho.cpu().numpy().reshape(prob.mesh.ncells, q ** 3)
        assert rel_fro(got, rho_ref) < 1e-6
        rho64 = torch.empty_like(rho)
        ctx.density(torch.tensor(x32.astype(np.float64), device=DEV), rho64,
                    torch.tensor(f32.astype(np.float64), device=DEV), occ, prec="fp64")
        assert rel_fro(got, rho64.cpu().numpy().reshape(prob.mesh.ncells, q ** 3)) < 1e-6
        # one column: a single ragged chunk, no partially occupied block
        ctx.density(torch.tensor(x32[:, :1].copy(), device=DEV), rho, prec="mixed")
        got1 = rho.cpu().numpy().reshape(prob.mesh.ncells, q ** 3)
        assert rel_fro(got1, od.density(prob, x32[:, :1].astype(np.float64))) < 1e-6
    finally:
        ctx.destroy()
