"""The input generators and the test-side exact-length routine (CPU).

The GPU tests check tours that the device built with tests/gpu_common.exact_tour_lengths, a
routine written independently of the oracle; here the two are checked against each other on
synthetic tours (including coincident cities and an edge below the 2^-96 grid), and the
spatially coherent tours that the full-size replay loads on both sides are checked to be
seeded permutations."""
import numpy as np
import pytest

import aco_synth
import oracle

pytest.importorskip("torch")  # tests.gpu_common imports torch
from tests.gpu_common import exact_tour_lengths  # noqa: E402


@pytest.mark.parametrize("n", [3, 10, 1000, 20000])
def test_exact_tour_lengths_agree_with_the_oracle(n):
    xy = aco_synth.clustered(n, 5, 0.01, n)
    tours = aco_synth.permutations(4, n, n)
    assert np.array_equal(exact_tour_lengths(xy, tours), oracle.tour_lengths(xy, tours))


def test_exact_tour_lengths_degenerate_edges():
    xy = np.array([[0.0, 0.0], [0.0, 0.0], [1e-20, 0.0], [1.0, 1.0], [0.5, 2.0]])
    tours = np.array([[0, 1, 2, 3, 4], [4, 3, 2, 1, 0], [2, 0, 4, 1, 3]], np.int32)
    assert np.array_equal(exact_tour_lengths(xy, tours), oracle.tour_lengths(xy, tours))


def test_snake_tours_are_seeded_permutations():
    xy = aco_synth.clustered(5000, 20, 0.01, 3)
    a = aco_synth.snake_tours(xy, 6, 7, grid=64, reversals=16, max_len=300)
    b = aco_synth.snake_tours(xy, 6, 7, grid=64, reversals=16, max_len=300)
    c = aco_synth.snake_tours(xy, 6, 8, grid=64, reversals=16, max_len=300)
    assert a.dtype == np.int32 and a.shape == (6, 5000)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    for t in a:
        assert np.array_equal(np.sort(t), np.arange(5000))
    # spatially coherent: far shorter than random permutations of the same cities
    rand = aco_synth.permutations(6, 5000, 1)
    assert oracle.tour_lengths(xy, a).max() < 0.2 * oracle.tour_lengths(xy, rand).min()


def test_oracle_pool_gives_the_oracles_initial_tours():
    """The spawn pool used by the full-size parity test returns what one oracle builds itself."""
    from tests import oracle_pool

    xy = aco_synth.clustered(300, 4, 0.05, 8)
    p = dict(mode=1, n=300, m=12, k=8, alpha=1.0, beta=2.0, tau0=1.0, max_mod_frac=0.3, p_partial=1.0, seed=4)
    cand = oracle.knn(xy, 8)
    got = oracle_pool.initial_tours(xy, cand, p, [3, 7, 11], workers=2)
    ref = oracle.Oracle(xy, cand=cand, **p)
    ref.construct(0)
    for a in (3, 7, 11):
        assert np.array_equal(got[a][0], ref.newtours[a])
        assert got[a][1] == ref.newlen[a]
