"""One ChFSI iteration on a host-resident block through the C ABI
(chfsi_step_host): the result written back into host memory equals the same
iteration run on a device-resident block, bit for bit, whichever moves the
rows (the SMs over the host link, or the copy engines), and for pinned and
pageable host buffers (on a Grace host the GPU may reach pageable memory
directly; the library then uses the SM copies for it as well)."""
import numpy as np
import pytest
import torch

from paper_1903_10959_gb300 import ChfsiError, workloads as W

from gpu_util import gpu_context

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("prec", ["bf16x3", "fp64", "f16x2"])
def test_step_host_equals_device_step(prec):
    s = W.small_periodic(seed=81, ncell=3, p=4, L=7.5, n_wells=3, n_want=20, degree=10, iters=2)
    ctx = gpu_context(s)
    try:
        M, n = ctx.ndofs, s.n_sub
        dt = torch.float64 if prec == "fp64" else torch.float32
        x0 = torch.tensor(W.start_block(s.seed, M, n)).to(dt)
        b = ctx.bounds(20, s.seed)
        Xd = x0.to(DEV)
        ctx.cholgs(Xd, prec=prec)
        D = ctx.rayleigh_ritz(Xd, prec=prec)
        a, a0 = float(D[-1]), float(D[0])
        start = Xd.cpu()
        # reference: the same iteration on the device-resident block
        Xr = start.to(DEV)
        ctx.filter(Xr, s.degree, a, b, a0, prec=prec)
        ctx.cholgs(Xr, prec=prec)
        Dr = ctx.rayleigh_ritz(Xr, prec=prec)
        ref = Xr.cpu()
        for mode, pinned in [(0, True), (1, True), (2, True), (0, False)]:
            Xh = start.clone().pin_memory() if pinned else start.clone()
            work = torch.empty_like(Xd)
            ev, ms = ctx.step_host(Xh, work, s.degree, a, b, a0, prec=prec, copy_mode=mode)
            assert torch.equal(Xh, ref), (mode, pinned)
            assert np.array_equal(ev, Dr)
            assert np.all(ms >= 0) and ms[1] > 0
        # SM copies need a device-mapped host block: a pageable one is refused,
        # unless the GPU reaches pageable memory directly (coherent host link),
        # in which case the result is the same
        Xp = start.clone()
        try:
            ctx.step_host(Xp, torch.empty_like(Xd), s.degree, a, b, a0, prec=prec, copy_mode=2)
        except ChfsiError as err:
            assert err.status == 1
        else:
            assert torch.equal(Xp, ref)
    finally:
        ctx.destroy()
