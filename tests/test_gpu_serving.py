"""Serving loop on the GPU: continuous batching (admitted requests overlap on
the device), admission by the device-memory budget, warm-started re-solves,
and the same result for a request alone and in the mix."""
import dataclasses
import time

import numpy as np
import pytest

from paper_1903_10959_gb300 import Server, workloads as W
from tests.gpu_util import oracle_problem

pytestmark = pytest.mark.gpu

DEGREE, ITERS, WARM = 20, 24, 6


def _mesh(s):
    return ((s.ncell,) * 3, (s.L,) * 3, s.p, s.periodic)


@pytest.fixture(scope="module")
def small():
    """A 1,000-unknown request whose wanted count ends at a spectral gap of the
    oracle's dense spectrum (the cut through a near-degenerate cluster would
    leave its members unconverged at any precision), with the exact spectra
    of all of its potentials."""
    (s, seq), = W.serving_requests(seed=12, count=1, dof_range=(1.0e3, 3.4e3), n_range=(12, 40),
                                   degree=DEGREE, resolves=2)
    exact = [np.linalg.eigvalsh(oracle_problem(dataclasses.replace(s, depths=d)).dense_Htilde())
             for d in [s.depths] + list(seq)]
    gaps = np.diff(exact[0][:s.n_want + 1])
    k = 1 + max(i for i in range(len(gaps)) if gaps[i] > 0.1)
    return dataclasses.replace(s, n_want=k), seq, exact


@pytest.fixture(scope="module")
def requests(small):
    s, seq, _ = small
    return [(s, seq)] + W.serving_requests(seed=11, count=3, dof_range=(3.0e3, 2.5e4),
                                           n_range=(12, 40), degree=DEGREE, resolves=2)


def _run(requests, max_active, budget=1 << 36, prec="mixed", tol=0.0, iters=ITERS, warm=WARM,
         polish=0):
    out, t_sub = [], []
    with Server(budget, max_active) as sv:
        tickets = []
        for s, seq in requests:
            t_sub.append(time.perf_counter())
            tickets.append(sv.submit(_mesh(s), s.n_sub, s.centres, s.depths, s.widths,
                                     depth_seq=seq, degree=s.degree, iters=iters,
                                     warm_iters=warm, tol=tol, n_check=s.n_want, prec=prec,
                                     seed=s.seed, polish_iters=polish))
        for t in tickets:
            out.append(sv.poll(t, wait=True))
    for r, t0 in zip(out, t_sub):
        r["admit"] = t0 + r["queue_ms"] * 1e-3
        r["end"] = t0 + r["total_ms"] * 1e-3
    return out


@pytest.fixture(scope="module")
def mix(requests):
    return _run(requests, max_active=4)


@pytest.fixture(scope="module")
def alone(requests):
    return _run(requests, max_active=1)


def test_all_requests_succeed(mix, requests):
    for r, (s, seq) in zip(mix, requests):
        assert r["status"] == 0, r["error"]
        assert r["nsolves"] == len(seq) + 1
        assert r["used_bytes"] <= r["est_bytes"]


def test_mix_overlaps_on_the_device(mix):
    """Every request is admitted before the first one finishes."""
    first_end = min(r["end"] for r in mix)
    assert all(r["admit"] < first_end for r in mix)


def test_alone_requests_run_one_at_a_time(alone):
    order = sorted(alone, key=lambda r: r["admit"])
    for a, b in zip(order, order[1:]):
        assert b["admit"] >= a["end"] - 2e-3


def test_alone_equals_mix(mix, alone):
    """Requests share no device data and every reduction has a fixed order, so
    each result is bit-identical alone and in the mix."""
    for a, m in zip(alone, mix):
        assert np.array_equal(a["evals"], m["evals"])
        assert a["max_gresidual"] == m["max_gresidual"]


MIXED_GRES_FLOOR = 5e-6


def test_eigenvalues_match_dense_oracle(mix, small):
    """Every solve of the small request (original and perturbed potentials)
    against the oracle's dense diagonalisation of H~: <= 1e-7 Ha on the wanted
    pairs.  The generalized residual of vectors filtered in binary32 / 3xTF32
    stalls at a few 1e-6 (each degree step adds ~sqrt(n_e) * 2^-22 relative
    noise to the block, and binary32 storage alone gives ~3e-7), so the mixed
    residual is held to that floor; the binary64 path reaches 1e-8 below."""
    s, seq, exact = small
    r = mix[0]
    for j in range(len(seq) + 1):
        err = np.abs(r["evals"][j][:s.n_want] - exact[j][:s.n_want]).max()
        assert err < 1e-7, (j, err)
        assert r["max_gresidual"][j] < MIXED_GRES_FLOOR, (j, r["max_gresidual"][j])


POLISHED_GRES = 1e-6


@pytest.mark.parametrize("prec", ["mixed", "bf16x3", "f16x2"])
def test_polished_solves_meet_the_residual_target(small, prec):
    """With the binary64 polish (one binary64 iteration of the request's
    degree after the mixed iterations, chfsi_solve_polish) every solve of the
    small request -- cold and warm, original and perturbed potentials --
    meets the generalized-residual target <= 1e-6 and <= 1e-7 Ha against the
    oracle's dense diagonalisation."""
    s, seq, exact = small
    r, = _run([(s, seq)], max_active=1, prec=prec, polish=1)
    assert r["status"] == 0, r["error"]
    for j in range(len(seq) + 1):
        assert r["max_gresidual"][j] <= POLISHED_GRES, (j, r["max_gresidual"][j])
        err = np.abs(r["evals"][j][:s.n_want] - exact[j][:s.n_want]).max()
        assert err <= 1e-7, (j, err)


def test_budget_admits_one_at_a_time(requests):
    """A budget that fits only the largest request once serialises them:
    later requests wait in the queue until memory frees up."""
    big = max(Server.estimate(_mesh(s), s.n_sub, nwells=len(s.depths)) for s, _ in requests)
    res = _run(requests[:3], max_active=3, budget=int(big * 1.05), iters=4, warm=1)
    assert all(r["status"] == 0 for r in res)
    order = sorted(res, key=lambda r: r["admit"])
    for a, b in zip(order, order[1:]):
        assert b["admit"] >= a["end"] - 2e-3
    assert max(r["queue_ms"] for r in res) > 0.5 * min(r["total_ms"] for r in res)


def test_warm_start_needs_fewer_iterations(small):
    """FP64 with a residual tolerance: the re-solves from the previous
    eigenvectors stop after fewer ChFSI iterations than the cold solve."""
    s, seq, exact = small
    r, = _run([(s, seq)], max_active=1, prec="fp64", tol=1e-8, iters=60, warm=60)
    assert r["status"] == 0, r["error"]
    assert r["iters"][0] < 60
    assert max(r["iters"][1:]) < r["iters"][0]
    assert max(r["max_gresidual"]) < 1e-8
    for j in range(len(seq) + 1):
        assert np.abs(r["evals"][j][:s.n_want] - exact[j][:s.n_want]).max() < 1e-10
