"""Pins of the oracle's Independent Roulette (Section 3's selection rule; §8(f) F2).

Independent Roulette gives each candidate its own uniform draw and takes the largest weight x
draw.  For two candidates with weights w1 >= w2 the first wins with probability 1 - w2 / (2 w1)
(the area of {w1 u1 > w2 u2} in the unit square); equal weights give a uniform choice; a zero
weight is never picked."""
import math

import numpy as np

import aco_synth
import oracle


def _freq(w, draws=20000, seed=7):
    picks = np.array([oracle.ir_pick(w, seed, t, 3, 5) for t in range(draws)])
    return np.array([(picks == r).mean() for r in range(len(w))]), picks


def test_two_candidates_closed_form():
    for w1, w2 in [(1.0, 0.5), (2.0, 1.9), (3.0, 0.3)]:
        f, _ = _freq([w1, w2])
        p = 1.0 - w2 / (2.0 * w1)
        sigma = math.sqrt(p * (1 - p) / 20000)
        assert abs(f[0] - p) < 5 * sigma, (w1, w2, f[0], p)
        f, _ = _freq([w2, w1])  # order does not matter
        assert abs(f[1] - p) < 5 * sigma


def test_equal_weights_uniform_and_zero_never_picked():
    f, picks = _freq([1.0, 0.0, 1.0, 1.0, 0.0])
    assert np.all(f[[1, 4]] == 0.0)
    assert np.all(np.abs(f[[0, 2, 3]] - 1 / 3) < 5 * math.sqrt((1 / 3) * (2 / 3) / 20000))
    assert oracle.ir_pick([0.0, 0.0], 1, 0, 0, 0) == -1
    assert oracle.ir_pick([0.25], 1, 0, 0, 0) == 0


def test_ir_is_not_the_eq1_wheel():
    # Eq. 1 would pick the first of (1, 0.5) with probability 2/3; IR does so with 3/4
    f, _ = _freq([1.0, 0.5])
    assert abs(f[0] - 0.75) < 0.015 and abs(f[0] - 2 / 3) > 0.05


def test_ir_colony_finds_the_optimum_of_small_instances():
    import itertools

    for seed in (1, 2):
        xy = aco_synth.uniform(8, 40 + seed)
        best = min(oracle.tour_length(xy, np.array((0,) + p)) for p in itertools.permutations(range(1, 8)))
        col = oracle.Oracle(xy, mode=1, n=8, m=8, k=5, max_mod_frac=1.0, seed=seed, selection=1)
        for it in range(30):
            col.iterate(it)
        assert col.clen.min() >= best - 1e-12
        assert col.clen.min() <= best * (1 + 1e-12)
        for t in col.lbest:
            assert sorted(t) == list(range(8))
