"""Pins of the CPU oracle to what the paper and mathematics fix (no GPU).

Each test checks the oracle against something other than itself: published known-answer
vectors, a worked example of Eq. 1, closed forms (Eq. 2 scaling, the Eq. 3-5 deposit total,
the n(n-1)/2 scan count of a full construction), brute force on tiny inputs (the exhaustive TSP
optimum, nearest-neighbour tours, candidate lists by sorting) and statistical agreement of the
wheel with Eq. 1's probabilities.
"""
import itertools
import math
import os

import numpy as np
import pytest

import aco_synth
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ------------------------------------------------------------------ random numbers
def test_philox_known_answers():
    for r in _rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_u53_and_bounded_closed_forms():
    assert oracle.u53(0, 0) == 0.0
    assert oracle.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle.u53(0x80000000, 0) == 0.5
    assert oracle.bounded(0, 100) == 0
    assert oracle.bounded(0xFFFFFFFF, 100) == 99
    assert oracle.bounded(0x80000000, 10) == 5
    assert oracle.powr(3.0, 2.0) == 9.0 and oracle.powr(2.0, 0.0) == 1.0
    assert oracle.powr(2.0, 0.5) == math.sqrt(2.0)


# ------------------------------------------------------------------ lengths and candidates
def _py_edge(xy, i, j):
    dx = xy[i, 0] - xy[j, 0]
    dy = xy[i, 1] - xy[j, 1]
    return math.sqrt(dx * dx + dy * dy)


@pytest.mark.parametrize("n,seed", [(3, 1), (50, 2), (1000, 3)])
def test_tour_length_is_correctly_rounded_sum(n, seed):
    """Length = correctly rounded exact sum of the FP64 edge lengths (math.fsum is exact)."""
    xy = aco_synth.uniform(n, seed)
    rng = np.random.default_rng(seed)
    for _ in range(5):
        t = rng.permutation(n).astype(np.int32)
        ref = math.fsum(_py_edge(xy, int(t[p]), int(t[(p + 1) % n])) for p in range(n))
        assert oracle.tour_length(xy, t) == ref
        # order independence: rotation and reversal give the same bits
        assert oracle.tour_length(xy, np.roll(t, 7)) == ref
        assert oracle.tour_length(xy, t[::-1].copy()) == ref


def test_tour_length_square():
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float64)
    assert oracle.tour_length(xy, np.array([0, 1, 2, 3], np.int32)) == 4.0
    assert oracle.tour_length(xy, np.array([0, 2, 1, 3], np.int32)) == 2.0 + 2.0 * math.sqrt(2.0)


@pytest.mark.parametrize("gen,k", [("uniform", 8), ("clustered", 16), ("grid", 6)])
def test_knn_matches_sorting(gen, k):
    if gen == "uniform":
        xy = aco_synth.uniform(600, 5)
    elif gen == "clustered":
        xy = aco_synth.clustered(600, 7, 0.01, 6)
    else:  # integer lattice: many exact distance ties, broken by index
        g = np.arange(20, dtype=np.float64)
        xy = np.ascontiguousarray(np.stack(np.meshgrid(g, g), -1).reshape(-1, 2))
    n = xy.shape[0]
    cand = oracle.knn(xy, k)
    d2 = ((xy[:, None, :] - xy[None, :, :]) ** 2).sum(-1)  # exact for these inputs? only used via lexsort below
    for i in range(0, n, 7):
        dx = xy[i, 0] - xy[:, 0]
        dy = xy[i, 1] - xy[:, 1]
        key = dx * dx + dy * dy
        order = np.lexsort((np.arange(n), key))
        order = order[order != i][:k]
        assert np.array_equal(cand[i], order), i
    del d2


def test_knn_rejects_coincident_cities():
    xy = np.array([[0, 0], [1, 0], [0, 0], [0, 1]], np.float64)
    with pytest.raises(ValueError):
        oracle.knn(xy, 2)


# ------------------------------------------------------------------ Eq. 1
def test_eq1_unit_square_worked_example():
    rows = _rows("eq1_unit_square.txt")
    xy = np.array([[float(r[1]), float(r[2])] for r in rows[:4]], np.float64)
    expect = [float(x) for x in rows[4]]
    o = oracle.Oracle(xy, mode=oracle.MODE_DENSE, n=4, m=1, alpha=1.0, beta=2.0, rho=0.5, tau0=1.0)
    p, _ = o.step_probs(0, np.array([1, 0, 0, 0], np.uint8))
    assert p[0] == 0.0
    assert np.allclose(p[1:], expect, rtol=0, atol=1e-15)
    assert abs(p.sum() - 1.0) < 1e-15


def test_eq1_alpha_zero_is_heuristic_only():
    xy = aco_synth.uniform(30, 9)
    o = oracle.Oracle(xy, mode=oracle.MODE_DENSE, n=30, m=1, alpha=0.0, beta=2.0, rho=0.5, tau0=1.0)
    vis = np.zeros(30, np.uint8)
    vis[[0, 4, 9]] = 1
    p1, _ = o.step_probs(0, vis)
    rng = np.random.default_rng(3)
    o.set_tau(rng.uniform(0.1, 10.0, (30, 30)))
    p2, _ = o.step_probs(0, vis)
    assert np.array_equal(p1, p2)
    eta2 = np.array([0.0 if vis[j] else 1.0 / (_py_edge(xy, 0, j) ** 2) for j in range(30)])
    assert np.allclose(p1, eta2 / eta2.sum(), rtol=1e-12, atol=0)


def test_eq1_pheromone_scales_probability():
    """With beta = 0, p is proportional to tau^alpha: doubling one tau doubles its odds."""
    xy = aco_synth.uniform(6, 4)
    o = oracle.Oracle(xy, mode=oracle.MODE_DENSE, n=6, m=1, alpha=1.0, beta=0.0, rho=0.5, tau0=1.0)
    tau = np.ones((6, 6))
    tau[0, 3] = 2.0
    o.set_tau(tau)
    p, _ = o.step_probs(0, np.array([1, 0, 0, 0, 0, 0], np.uint8))
    assert np.allclose(p, [0, 1 / 6, 1 / 6, 2 / 6, 1 / 6, 1 / 6], atol=1e-15)


def test_wheel_frequencies_follow_eq1():
    """First decisions of many ants from the same city follow Eq. 1 (chi-square)."""
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1], [0.5, 2.0]], np.float64)
    n, m = 5, 40000
    o = oracle.Oracle(xy, mode=oracle.MODE_DENSE, n=n, m=m, alpha=1.0, beta=2.0, rho=0.5, tau0=1.0, seed=77)
    o.construct(0)
    T = o.newtours
    for start in range(n):
        sel = T[T[:, 0] == start, 1]
        vis = np.zeros(n, np.uint8)
        vis[start] = 1
        p, _ = o.step_probs(start, vis)
        counts = np.bincount(sel, minlength=n).astype(float)
        exp = p * sel.size
        mask = exp > 0
        chi2 = (((counts - exp) ** 2)[mask] / exp[mask]).sum()
        assert counts[start] == 0
        assert chi2 < 25.0, (start, counts, exp)  # 3 dof; P(chi2 > 25) ~ 1.5e-5


# ------------------------------------------------------------------ Eq. 2-5 (dense)
def _dense_run(n=12, m=7, seed=5, rho=0.3):
    xy = aco_synth.uniform(n, seed)
    o = oracle.Oracle(xy, mode=oracle.MODE_DENSE, n=n, m=m, alpha=1.0, beta=2.0, rho=rho, tau0=1.0, seed=seed)
    return xy, o


def test_eq2_evaporation_exact_and_eq3_deposit_sums():
    xy, o = _dense_run()
    n, m, rho = 12, 7, 0.3
    rng = np.random.default_rng(1)
    tau0 = rng.uniform(0.5, 3.0, (n, n))
    tau0 = (tau0 + tau0.T) / 2
    o.set_tau(tau0)
    o.construct(3)
    T = o.newtours
    C = o.newlen
    o.update()
    tau1 = o.tau
    # brute-force edge membership of every tour
    member = np.zeros((m, n, n), bool)
    for a in range(m):
        for p in range(n):
            i, j = T[a, p], T[a, (p + 1) % n]
            member[a, i, j] = member[a, j, i] = True
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            ev = (1.0 - rho) * tau0[i, j]
            if not member[:, i, j].any():
                assert tau1[i, j] == ev  # Eq. 2 alone, bit-exact
            else:
                dep = sum(1.0 / C[a] for a in range(m) if member[a, i, j])
                assert abs(tau1[i, j] - (ev + dep)) <= 4e-16 * (ev + dep)
    # total deposit over undirected edges = sum_k n / C_k (each tour has n edges)
    iu = np.triu_indices(n, 1)
    total = (tau1 - (1.0 - rho) * tau0)[iu].sum()
    assert abs(total - sum(n / C[a] for a in range(m))) < 1e-12
    assert np.array_equal(tau1, tau1.T)


def test_full_construction_scans_triangle_number():
    """A full tour evaluates n-1, n-2, ..., 1 unvisited cities: n(n-1)/2 (the paper's
    triangle-number cost argument, Section 5)."""
    n, m = 40, 3
    xy, o = _dense_run(n=n, m=m)
    o.reset_counters()
    o.construct(0)
    c = o.counters()
    assert c["decisions"] == m * (n - 1)
    assert c["scans"] == m * n * (n - 1) // 2


def test_tours_are_permutations_dense():
    xy, o = _dense_run(n=30, m=10)
    for it in range(5):
        o.iterate(it)
        T = o.newtours
        assert all(np.array_equal(np.sort(t), np.arange(30)) for t in T)
        assert np.array_equal(o.newlen, oracle.tour_lengths(xy, T))


# ------------------------------------------------------------------ exhaustive optimum
def _optimum(xy):
    n = xy.shape[0]
    best = math.inf
    for perm in itertools.permutations(range(1, n)):
        if perm[0] > perm[-1]:
            continue
        t = np.array((0,) + perm, np.int32)
        best = min(best, oracle.tour_length(xy, t))
    return best


@pytest.mark.parametrize("n", [6, 8, 9])
def test_dense_reaches_exhaustive_optimum(n):
    xy = aco_synth.uniform(n, 100 + n)
    opt = _optimum(xy)
    o = oracle.Oracle(xy, mode=oracle.MODE_DENSE, n=n, m=10, alpha=1.0, beta=2.0, rho=0.5, tau0=1.0, seed=n)
    best = math.inf
    for it in range(30):
        o.iterate(it)
        best = min(best, o.newlen.min())
        assert o.newlen.min() >= opt * (1 - 1e-15)
    assert best == opt


@pytest.mark.parametrize("n", [7, 9])
def test_partialaco_reaches_exhaustive_optimum(n):
    xy = aco_synth.clustered(n, 2, 0.3, 200 + n)
    opt = _optimum(xy)
    o = oracle.Oracle(xy, mode=oracle.MODE_LBEST, n=n, m=6, k=3, alpha=1.0, beta=2.0, tau0=1.0,
                      max_mod_frac=1.0, seed=n)
    for it in range(60):
        o.iterate(it)
        assert o.clen.min() >= opt * (1 - 1e-15)
    assert o.clen.min() == opt


# ------------------------------------------------------------------ Section 3 / Algorithm 1
def _nn_tour(xy, start):
    n = xy.shape[0]
    vis = np.zeros(n, bool)
    t = [start]
    vis[start] = True
    for _ in range(n - 1):
        i = t[-1]
        best, bd = -1, math.inf
        for j in range(n):
            if not vis[j]:
                dx = xy[i, 0] - xy[j, 0]
                dy = xy[i, 1] - xy[j, 1]
                d2 = dx * dx + dy * dy
                if d2 < bd:
                    best, bd = j, d2
        t.append(best)
        vis[best] = True
    return np.array(t, np.int32)


def test_k1_initial_tours_are_nearest_neighbour_tours():
    """With one candidate and tau = tau0 (no l_best yet), Eq. 1 over the list always takes the
    nearest city and the exhausted-list rule takes the nearest unvisited one: the initial tour
    is the greedy nearest-neighbour tour from the drawn start."""
    xy = aco_synth.uniform(80, 21)
    o = oracle.Oracle(xy, mode=oracle.MODE_LBEST, n=80, m=5, k=1, seed=4)
    o.construct(0)
    for t in o.newtours:
        assert np.array_equal(t, _nn_tour(xy, int(t[0])))


def _lbest_colony(n=60, m=8, k=6, f=0.3, seed=11, p_partial=1.0):
    xy = aco_synth.clustered(n, 3, 0.05, seed)
    o = oracle.Oracle(xy, mode=oracle.MODE_LBEST, n=n, m=m, k=k, alpha=1.0, beta=2.0, tau0=1.0,
                      max_mod_frac=f, p_partial=p_partial, seed=seed)
    return xy, o


def test_partialaco_invariants():
    n, m, f = 60, 8, 0.3
    xy, o = _lbest_colony(n=n, m=m, f=f)
    o.iterate(0)
    prev_c = o.clen
    assert np.array_equal(prev_c, oracle.tour_lengths(xy, o.lbest))
    fm = math.floor(f * n)
    for it in range(1, 25):
        L = o.lbest
        o.construct(it)
        T = o.newtours
        s, M = o.segments()
        for a in range(m):
            assert 1 <= M[a] <= fm
            P = n - M[a]
            keep = [(s[a] + q) % n for q in range(P)]
            assert np.array_equal(T[a, keep], L[a, keep])  # the preserved part is untouched
            assert np.array_equal(np.sort(T[a]), np.arange(n))
        assert np.array_equal(o.newlen, oracle.tour_lengths(xy, T))
        o.update()
        c = o.clen
        assert np.all(c <= prev_c)  # l_best never gets longer
        better = o.newlen < prev_c
        assert np.array_equal(o.lbest[better], T[better])
        assert np.array_equal(o.lbest[~better], L[~better])
        prev_c = c


def test_pheromone_weights_brute_force():
    """Q[i][r] = sum over ants with edge (i, cand[i][r]) in l_best of round(C_g/C_a * 2^32),
    checked against a dense scatter of every l_best edge; w = C_g/C_a is in (0, 1]."""
    n, m, k = 60, 8, 6
    xy, o = _lbest_colony(n=n, m=m, k=k)
    for it in range(6):
        o.iterate(it)
    W, Q, q = o.cand_weights()
    L, C = o.lbest, o.clen
    cg = C.min()
    w = cg / C
    assert np.all(w > 0) and np.all(w <= 1) and w[np.argmin(C)] == 1.0
    assert np.array_equal(q, np.array([round(x * 2 ** 32) for x in w], np.uint64))
    dense = np.zeros((n, n), np.uint64)
    for a in range(m):
        for p in range(n):
            i, j = L[a, p], L[a, (p + 1) % n]
            dense[i, j] += q[a]
            dense[j, i] += q[a]
    cand = o.cand
    assert np.array_equal(Q, dense[np.arange(n)[:, None], cand])
    etab = o.etab
    tau = 1.0 + Q.astype(np.float64) * 2.0 ** -32
    assert np.array_equal(W, tau * etab)


def test_partial_probability_zero_builds_full_tours():
    n, m = 40, 6
    xy, o = _lbest_colony(n=n, m=m, p_partial=0.0)
    o.iterate(0)
    o.construct(1)
    s, M = o.segments()
    assert np.all(s == -1) and np.all(M == n - 1)


def test_lbest_step_probs_candidate_form():
    """Eq. 1 over the candidate list: unvisited candidates only, sums to one."""
    xy, o = _lbest_colony()
    o.iterate(0)
    vis = np.zeros(60, np.uint8)
    vis[:20] = 1
    p, ex = o.step_probs(30, vis)
    cand = o.cand[30]
    assert not ex
    assert np.all(p[vis[cand] == 1] == 0)
    assert abs(p.sum() - 1) < 1e-15


@pytest.mark.parametrize("gen", ["uniform", "clustered", "lattice"])
def test_knn_sweep_and_single_query_match_definition(gen):
    if gen == "uniform":
        xy = aco_synth.uniform(700, 31)
    elif gen == "clustered":
        xy = aco_synth.clustered(700, 5, 0.02, 32)
    else:
        g = np.arange(25, dtype=np.float64)
        xy = np.ascontiguousarray(np.stack(np.meshgrid(g, g), -1).reshape(-1, 2))
    k = 12
    ref = oracle.knn(xy, k)
    assert np.array_equal(oracle.knn_sweep(xy, k), ref)
    for i in range(0, xy.shape[0], 37):
        assert np.array_equal(oracle.knn_one(xy, k, i), ref[i])


def test_oracle_with_supplied_candidates_is_identical():
    xy = aco_synth.clustered(120, 3, 0.05, 8)
    kw = dict(mode=oracle.MODE_LBEST, n=120, m=6, k=7, max_mod_frac=0.4, seed=3)
    a = oracle.Oracle(xy, **kw)
    b = oracle.Oracle(xy, cand=oracle.knn_sweep(xy, 7), **kw)
    for it in range(8):
        a.iterate(it)
        b.iterate(it)
    assert np.array_equal(a.lbest, b.lbest) and np.array_equal(a.clen, b.clen)


@pytest.mark.parametrize("p_partial,fallback", [(1.0, 0), (0.6, 1)])
def test_threaded_construction_equals_sequential(p_partial, fallback):
    """Ants spread over host threads build the same tours with the same counters."""
    n, m = 400, 24
    xy = aco_synth.clustered(n, 5, 0.03, 19)
    kw = dict(mode=oracle.MODE_LBEST, n=n, m=m, k=8, max_mod_frac=0.3, p_partial=p_partial, seed=19,
              fallback=fallback)
    a, b = oracle.Oracle(xy, **kw), oracle.Oracle(xy, **kw)
    for it in range(5):
        a.construct(it)
        b.construct(it, threads=5)
        assert np.array_equal(a.newtours, b.newtours) and np.array_equal(a.newlen, b.newlen)
        assert a.counters() == b.counters()
        a.update()
        b.update()
    sub = np.array([3, 17, 5, 22], np.int32)
    a.construct(5, ants=sub)
    b.construct(5, ants=sub, threads=3)
    assert np.array_equal(a.newtours[sub], b.newtours[sub])
