"""Pins of the oracle's exhausted-list rule with pheromone on edges outside the candidate lists.

When every candidate of the current city is visited, the ant falls back to the ordinary rule over
all unvisited cities (Section 6), and the pheromone of an edge outside the candidate lists still
comes from the whole l_best population (Section 3).  The values below were worked by hand
(tests/golden/exhausted_step_six_cities.txt): a six-city instance whose two l_best tours have
integer lengths 20 and 28, so every pheromone value is 1, 1 + omega or 2 + omega with
omega = round(20/28 * 2^32) / 2^32.  A dropped predecessor side, a missing or inverted ant weight,
an unweighted count or a sum over one ant only changes these weights and probabilities.
"""
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "exhausted_step_six_cities.txt")


def _golden():
    xy, tours, queries = [], {}, []
    with open(GOLD) as f:
        for ln in f:
            if not ln.strip() or ln.startswith("#"):
                continue
            parts = ln.split()
            if parts[0] == "tour":
                tours[int(parts[1])] = [int(x) for x in parts[2:]]
            elif parts[0] == "query":
                head, probs, weights = ln.split("|")
                h = head.split()
                queries.append(dict(
                    name=h[1], city=int(h[2]), alpha=float(h[3]), argmax=int(h[4]),
                    visited=[int(x) for x in h[5].split(",")],
                    p={int(a): float(b) for a, b in (t.split(":") for t in probs.split())},
                    w={int(a): float(b) for a, b in (t.split(":") for t in weights.split())}))
            else:
                xy.append([float(parts[1]), float(parts[2])])
    return np.array(xy, np.float64), np.array([tours[0], tours[1]], np.int32), queries


def _colony(alpha, fallback):
    xy, tours, _ = _golden()
    o = oracle.Oracle(xy, mode=oracle.MODE_LBEST, n=6, m=2, k=1, alpha=alpha, beta=2.0, tau0=1.0, seed=1,
                      fallback=fallback)
    lens = oracle.tour_lengths(xy, tours)
    o.set_lbest(tours, lens)
    return o, lens


def test_instance_is_the_worked_one():
    xy, tours, _ = _golden()
    o, lens = _colony(1.0, 0)
    assert lens.tolist() == [20.0, 28.0]  # integer edge lengths, so the lengths are exact
    assert o.cand[:, 0].tolist() == [1, 0, 1, 4, 3, 4]  # nearest city, ties to the lower index


@pytest.mark.parametrize("fallback", [0, 1])
def test_weights_and_argmax_match_the_worked_values(fallback):
    _, _, queries = _golden()
    for q in queries:
        o, _ = _colony(q["alpha"], fallback)
        vis = np.zeros(6, np.uint8)
        vis[q["visited"]] = 1
        pick, w = o.exhausted_step(q["city"], vis, 0.0)
        for j in range(6):
            if vis[j]:
                assert w[j] == 0.0
            else:
                assert w[j] == pytest.approx(q["w"][j], rel=1e-14, abs=0), (q["name"], j)
        if fallback == 0:
            assert pick == q["argmax"], q["name"]
        ps = w / w.sum()
        for j, pj in q["p"].items():
            assert ps[j] == pytest.approx(pj, rel=1e-14, abs=0), (q["name"], j)


def test_boosted_city_beats_a_nearer_plain_city():
    """Queries b and d: the winner has pheromone and lies farther away than a city without any."""
    xy, _, queries = _golden()
    for name in ("b", "d"):
        q = next(x for x in queries if x["name"] == name)
        i, win = q["city"], q["argmax"]
        d = lambda j: np.hypot(*(xy[i] - xy[j]))  # noqa: E731
        plain = [j for j in q["w"] if j != win and d(j) < d(win)]
        assert plain, name


def test_boosted_counter():
    _, _, queries = _golden()
    o, _ = _colony(1.0, 0)
    o.reset_counters()
    for q in queries:
        if q["alpha"] != 1.0:
            continue
        vis = np.zeros(6, np.uint8)
        vis[q["visited"]] = 1
        o.exhausted_step(q["city"], vis, 0.0)
    assert o.counters()["boosted"] == 4  # every worked winner carries pheromone
    vis = np.array([1, 1, 1, 1, 0, 1], np.uint8)  # only city 4 is left; edge 1-4 is in no tour
    assert o.exhausted_step(1, vis, 0.0)[0] == 4
    assert o.counters()["boosted"] == 4


@pytest.mark.parametrize("name", ["a", "c", "e"])
def test_ordinary_rule_wheel_boundaries(name):
    """fallback = 1: the pick is the first unvisited city (index order) whose cumulative worked
    probability exceeds u, for u away from every boundary."""
    _, _, queries = _golden()
    q = next(x for x in queries if x["name"] == name)
    o, _ = _colony(q["alpha"], 1)
    vis = np.zeros(6, np.uint8)
    vis[q["visited"]] = 1
    js = sorted(q["p"])
    cum = np.cumsum([q["p"][j] for j in js])
    for u in np.linspace(0.0, 1.0 - 1e-9, 997):
        if np.min(np.abs(cum - u)) < 1e-9:
            continue
        want = js[int(np.searchsorted(cum, u, side="right"))]
        assert o.exhausted_step(q["city"], vis, float(u))[0] == want, (name, u)


def test_ordinary_rule_frequencies_chi_square():
    stats = pytest.importorskip("scipy.stats")
    _, _, queries = _golden()
    q = next(x for x in queries if x["name"] == "c")
    o, _ = _colony(1.0, 1)
    vis = np.zeros(6, np.uint8)
    vis[q["visited"]] = 1
    js = sorted(q["p"])
    counts = dict.fromkeys(js, 0)
    rng = np.random.default_rng(2017)
    draws = 20000
    for u in rng.random(draws):
        counts[o.exhausted_step(q["city"], vis, float(u))[0]] += 1
    obs = np.array([counts[j] for j in js], np.float64)
    exp = np.array([q["p"][j] for j in js]) * draws
    assert stats.chisquare(obs, exp).pvalue > 1e-4
