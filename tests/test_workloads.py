"""The seeded input recipe: the counter-based SplitMix64 generator against
the published sequence, its counter / stream / seed structure, and the
workload generators' documented shapes (the synthetic stand-ins for the
paper's crystals)."""
import numpy as np

from paper_1903_10959_gb300 import workloads as W


def test_splitmix64_matches_the_published_sequence():
    """SplitMix64 (Steele, Lea & Flood 2014) from state 0: the state advances
    by the golden gamma before each output; the first three outputs of the
    reference generator are these."""
    with np.errstate(over="ignore"):
        states = np.arange(1, 4, dtype=np.uint64) * W.GOLDEN
    out = [int(v) for v in W._finalize(states)]
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_based_draws():
    c = np.arange(1000, dtype=np.uint64)
    a = W.raw_u64(7, 1, c)
    # draw i depends only on (seed, stream, i): any subset regenerates the same values
    assert np.array_equal(W.raw_u64(7, 1, c[[5, 999, 0]]), a[[5, 999, 0]])
    assert not np.array_equal(W.raw_u64(7, 2, c), a)      # streams differ
    assert not np.array_equal(W.raw_u64(8, 1, c), a)      # seeds differ
    u = W.uniform_pm1(7, 1, np.arange(200000, dtype=np.uint64))
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 5e-3 and abs(u.var() - 1.0 / 3.0) < 5e-3


def test_start_block_rows_regenerate():
    X = W.start_block(3, 50, 17)
    rows = np.array([0, 13, 49])
    assert np.array_equal(W.start_block(3, rows, 17), X[rows])


def test_fcc_workload_shape():
    s = W.fcc_periodic()
    assert (s.ncell, s.p, s.L, s.degree) == (16, 6, 30.0, 40)
    assert s.ndofs == 884736 and s.n_want == 1000 and s.n_sub == 1100
    assert len(s.depths) == 256 and s.periodic
    assert np.all((s.depths >= 1.0) & (s.depths <= 3.0))
    assert np.all((s.widths >= 0.8) & (s.widths <= 1.2))
    # wells near the FCC sites of 4^3 conventional cells of side 7.5 (the lattice
    # shifted by a/4 along each axis), jittered by <= 0.3
    a = 7.5
    site = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) * a
    grid = np.array([[i, j, k] for k in range(4) for j in range(4) for i in range(4)]) * a
    sites = (grid[:, None, :] + site[None, :, :]).reshape(-1, 3) + 0.25 * a
    d = np.abs(((s.centres[:, None, :] - sites[None, :, :]) + 15.0) % 30.0 - 15.0).max(-1).min(1)
    assert d.max() <= 0.3 + 1e-12


def test_nonlocal_and_batched_workload_shapes():
    s = W.cubic_sites_nonlocal()
    assert (s.ncell, s.p, s.L, s.degree) == (20, 7, 40.0, 50)
    assert s.ndofs == 2744000 and s.n_want == 3000 and s.n_sub == 3300
    assert len(s.nl_centres) == 1000 and s.nl_h.shape == (1000, 4)
    assert np.all((s.nl_h >= 0.5) & (s.nl_h <= 2.0))
    sys = W.batched_systems()
    assert len(sys) == 64 and all(x.p == 5 and not x.periodic for x in sys)
    assert all(4 <= x.ncell <= 12 and 2 <= len(x.depths) <= 64 for x in sys)
    assert all(16 <= x.n_want <= 400 for x in sys)
