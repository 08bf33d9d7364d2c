"""Host logic of the serving loop that needs no GPU: the device-memory
estimate, argument checks and the admission rule for a request larger than
the whole budget (completed with ERR_OOM before anything touches a device)."""
import numpy as np
import pytest

from paper_1903_10959_gb300 import ChfsiError, Server, workloads as W
from paper_1903_10959_gb300._lib import STATUS


@pytest.fixture(scope="module")
def lib():
    from paper_1903_10959_gb300 import load
    try:
        return load()
    except RuntimeError as e:
        pytest.skip(str(e))


def _mesh(n, p):
    return ((n, n, n), (2.0 * n,) * 3, p, True)


def test_estimate_grows_with_size(lib):
    e1 = Server.estimate(_mesh(4, 5), 32)
    e2 = Server.estimate(_mesh(8, 5), 32)
    e3 = Server.estimate(_mesh(8, 5), 256)
    e4 = Server.estimate(_mesh(8, 5), 256, prec="fp64")
    assert 0 < e1 < e2 < e3
    M, n, ne = 40 ** 3, 256, 216
    assert e3 > M * n * 4 * 2 + 8 ** 3 * ne * ne * 8      # X, rotation scratch, binary64 cells
    assert e4 > M * n * 8 * 2 + 8 ** 3 * ne * ne * 8


def test_oversize_request_completes_with_oom(lib):
    (s, seq), = W.serving_requests(seed=3, count=1, dof_range=(3e3, 4e3), n_range=(8, 9),
                                   resolves=1)
    with Server(hbm_budget_bytes=1 << 20, max_active=2) as sv:
        t = sv.submit(((s.ncell,) * 3, (s.L,) * 3, s.p, True), s.n_sub, s.centres, s.depths,
                      s.widths, depth_seq=seq, degree=10, iters=2, warm_iters=1)
        r = sv.poll(t, wait=True)
    assert STATUS[r["status"]] == "ERR_OOM"
    assert r["nsolves"] == 0 and "budget" in r["error"]


def test_invalid_requests_are_rejected(lib):
    with Server(hbm_budget_bytes=1 << 30) as sv:
        mesh = _mesh(3, 5)
        c, d, w = np.zeros((2, 3)), np.ones(2), np.ones(2)
        with pytest.raises(ChfsiError):
            sv.submit(mesh, 0, c, d, w)                               # n < 1
        with pytest.raises(ChfsiError):
            sv.submit(mesh, 8, c, d, w, depth_seq=[d] * 16)           # > CHFSI_MAX_SOLVES
        with pytest.raises(ChfsiError):
            sv.submit(mesh, 8, c, d, w, degree=0)
        with pytest.raises(ChfsiError):
            sv.submit(mesh, 8, c, d, w, n_check=9)                    # more pairs than columns
    with pytest.raises(ChfsiError):
        Server(hbm_budget_bytes=0)


def test_serving_requests_shape():
    reqs = W.serving_requests(seed=5, count=64)
    dofs = np.array([s.ndofs for s, _ in reqs])
    assert dofs.min() >= 1.0e4 and dofs.max() <= 3.0e6
    assert {s.p for s, _ in reqs} == {5, 6, 7}
    for s, seq in reqs:
        assert len(seq) == 5 and all(q.shape == s.depths.shape for q in seq)
        rel = np.abs(np.array(seq) / s.depths - 1.0)
        assert rel.max() <= 0.01 * np.sqrt(3.0) + 1e-12 and rel.max() > 0
        assert 8 <= s.n_want <= max(8, s.ndofs // 8)
    t = W.poisson_arrivals(5, 4000, rate=2.0)
    assert np.all(np.diff(t) > 0) and abs(len(t) / t[-1] - 2.0) < 0.15
