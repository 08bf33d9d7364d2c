"""Filter lanes: the columns of a mixed-precision filter cut into groups of
whole 128-column tiles, each filtered on its own stream with its own scratch
(Eq. chebFilter acts on every column independently).  Every column must come
out bit-identical to the one-lane filter, for ragged widths, with and without
projectors, for both mixed precisions; a whole ChFSI solve as well."""
import numpy as np
import pytest
import torch

from paper_1903_10959_gb300 import ChfsiError, workloads as W

from gpu_util import gpu_context

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _sys(kind):
    if kind == "periodic":
        return W.small_periodic(seed=51, ncell=4, p=5, L=9.0, n_wells=5, n_want=20)
    s = W.small_periodic(seed=52, ncell=4, p=3, L=10.0, n_wells=6, n_want=16)
    s.nl_centres = s.centres[:3].copy()
    s.nl_h = 0.5 + np.arange(12).reshape(3, 4) / 8.0
    return s


@pytest.fixture(scope="module", params=["periodic", "nonlocal"])
def case(request):
    s = _sys(request.param)
    ctx = gpu_context(s)
    yield s, ctx
    ctx.set_filter_lanes(1)
    ctx.destroy()


@pytest.mark.parametrize("ncol", [129, 300, 700])
@pytest.mark.parametrize("prec", ["bf16x3", "mixed", "f16x2"])
def test_lanes_bit_identical(case, ncol, prec):
    s, ctx = case
    X0 = W.start_block(90 + ncol, ctx.ndofs, ncol).astype(np.float32)
    out = {}
    for lanes in (1, 2, 3, 4):
        ctx.set_filter_lanes(lanes)
        for block in (ncol, 200):
            ctx.set_blocking(block, 1)
            X = torch.tensor(X0, device=DEV)
            ctx.filter(X, 7, 4.0, 60.0, -3.0, prec=prec)
            out[(lanes, block)] = X.cpu()
    ctx.set_filter_lanes(1)
    for k, v in out.items():
        assert torch.equal(v, out[(1, ncol)]), k


def test_solve_with_lanes_equals_one_lane(case):
    s, ctx = case
    n = 260
    X0 = W.start_block(s.seed, ctx.ndofs, n).astype(np.float32)
    b = ctx.bounds(20, s.seed)
    res = []
    for lanes in (1, 2):
        ctx.set_filter_lanes(lanes)
        ctx.set_blocking(n, 1)
        X = torch.tensor(X0, device=DEV)
        D, _ = ctx.solve(X, 3, 10, b, prec="bf16x3")
        res.append((D, X.cpu()))
    ctx.set_filter_lanes(1)
    assert np.array_equal(res[0][0], res[1][0])
    assert torch.equal(res[0][1], res[1][1])


def test_bad_lane_count_is_rejected(case):
    s, ctx = case
    for bad in (0, 5):
        with pytest.raises(ChfsiError):
            ctx.set_filter_lanes(bad)
