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


def test_oracle_f_schedule_bounds_and_reduction():
    """F3: a growing f rebuilds at most floor(f(t) n) cities at iteration t; a constant schedule
    equals the fixed-f run."""
    from paper_1709_03187_gb300.colony import linear_f_schedule

    xy = aco_synth.clustered(400, 6, 0.03, 3)
    sched = linear_f_schedule(0.02, 0.3, 6)
    col = oracle.Oracle(xy, mode=1, n=400, m=10, k=8, max_mod_frac=0.3, seed=4)
    fixed = oracle.Oracle(xy, mode=1, n=400, m=10, k=8, max_mod_frac=0.3, seed=4)
    same = oracle.Oracle(xy, mode=1, n=400, m=10, k=8, max_mod_frac=0.3, seed=4)
    for it in range(8):
        col.set_max_mod_frac(sched(it))
        same.set_max_mod_frac(0.3)
        col.iterate(it)
        fixed.iterate(it)
        same.iterate(it)
        if it > 0:
            _, M = col.segments()
            assert np.all(M <= math.floor(sched(it) * 400))
    assert np.array_equal(same.lbest, fixed.lbest)
    assert not np.array_equal(col.lbest, fixed.lbest)
    # p_partial = 0: every ant builds a full tour
    col.set_p_partial(0.0)
    col.iterate(8)
    s, M = col.segments()
    assert np.all(s < 0)
