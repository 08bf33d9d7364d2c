"""Shared helpers of the GPU tests: oracle problems and library contexts for one System."""
import numpy as np


def oracle_problem(s):
    from oracle import hamiltonian as oham
    proj = None
    if len(s.nl_centres):
        proj = dict(centres=s.nl_centres, sigma=s.nl_sigma, rcut=s.nl_rcut, h=s.nl_h)
    return oham.wells_problem(s.ncell, s.p, s.L, s.periodic, s.centres, s.depths, s.widths,
                              projectors=proj)


def gpu_context(s, block=None):
    from paper_1903_10959_gb300 import Context
    ctx = Context(s.ncell, s.L, s.p, periodic=s.periodic)
    ctx.set_potential_gaussians(s.centres, s.depths, s.widths)
    if len(s.nl_centres):
        ctx.set_projectors(s.nl_centres, s.nl_h, s.nl_sigma, s.nl_rcut)
    ctx.build()
    if block:
        ctx.set_blocking(block, 32)
    return ctx


def rel_fro(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
