"""Pins of the oracle's windowed 2-opt (Section 3.2 local search, Section 5's 500-position
window; §8(f) F1).

2-opt replaces edges (a, b), (c, d) at tour positions i and j by (a, c), (b, d) when that
shortens the tour.  Pins: a crossed square is untangled to its perimeter; results are
permutations and never longer; at convergence no improving move within the window is left
(checked by brute force over every move the block passes can reach); with a window covering
the whole tour the result is a 2-opt local optimum for every non-wrapping move; in a colony,
the ants that draw local search get exactly their constructed tour improved."""
import numpy as np

import aco_synth
import oracle


def _gain(xy, T, i, j):
    d = lambda p, q: oracle.edge_len(xy, int(p), int(q))  # noqa: E731
    return (d(T[i], T[i + 1]) + d(T[j], T[j + 1])) - (d(T[i], T[j]) + d(T[i + 1], T[j + 1]))


def test_crossed_square_is_untangled():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    t, mv = oracle.two_opt_windowed(xy, np.array([0, 2, 1, 3]), window=10)
    assert mv == 1 and oracle.tour_length(xy, t) == 4.0
    assert sorted(t) == [0, 1, 2, 3]


def test_windowed_local_optimum_by_brute_force():
    for seed, W in [(1, 6), (2, 12), (3, 40)]:
        xy = aco_synth.clustered(150, 4, 0.05, seed)
        T0 = aco_synth.permutations(1, 150, seed)[0]
        T, mv = oracle.two_opt_windowed(xy, T0, W, max_passes=200)
        assert sorted(T) == list(range(150)) and mv > 0
        assert oracle.tour_length(xy, T) < oracle.tour_length(xy, T0)
        n = 150
        for i in range(n - 3):
            for j in range(i + 2, min(i + W - 2, n - 2) + 1):
                assert not _gain(xy, T, i, j) > 0.0, (seed, W, i, j)


def test_full_window_gives_a_2opt_local_optimum():
    xy = aco_synth.uniform(60, 5)
    T, _ = oracle.two_opt_windowed(xy, aco_synth.permutations(1, 60, 2)[0], window=60, max_passes=200)
    for i in range(60 - 3):
        for j in range(i + 2, 60 - 1):
            assert not _gain(xy, T, i, j) > 0.0


def test_local_search_in_a_colony():
    xy = aco_synth.clustered(300, 5, 0.03, 7)
    kw = dict(mode=1, n=300, m=12, k=8, max_mod_frac=0.5, seed=3)
    plain, ls = oracle.Oracle(xy, **kw), oracle.Oracle(xy, **kw)
    ls.set_local_search(1.0, 40)  # every ant draws local search; at most 8 per iteration
    plain.construct(0)
    ls.construct(0)
    a, b = plain.newtours, ls.newtours
    la, lb = plain.newlen, ls.newlen
    assert np.array_equal(a[8:], b[8:])           # ants 8.. are past the per-iteration cap
    assert np.all(lb[:8] <= la[:8]) and np.any(lb[:8] < la[:8])
    for a8 in range(8):
        t, _ = oracle.two_opt_windowed(xy, a[a8], 40)
        assert np.array_equal(t, b[a8])
    assert ls.ls_moves > 0
