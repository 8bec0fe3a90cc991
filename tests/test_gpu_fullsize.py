"""Parity at the benchmark's full size: 200,000 clustered cities, k = 16, m = 1024 ants, f = 1%.

The oracle cannot run the whole colony at this size in seconds, so it checks sampled outputs it
can compute one by one:
  * candidate lists of sampled cities by brute force (bit-exact);
  * initial tours (Algorithm 1, before its iterations) of eight sampled ants, built by the oracle from
    scratch with its own candidate lists, one host process each (bit-exact tours and lengths);
  * a PartialACO iteration of sampled ants from a synthetic l_best population (spatially coherent
    random tours from the input generators) loaded into both the colony and the oracle, each
    computing its own exact lengths;
and properties that hold at any size (permutations, exact lengths, l_best never lengthens,
C_gbest = min C_lbest, preserved part untouched, rebuilt count <= floor(f n)).
"""
import math

import numpy as np
import pytest

import aco_synth
import oracle
from tests import oracle_pool
from tests.gpu_common import exact_tour_lengths, require_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def colony200k():
    require_gpu()
    from paper_1709_03187_gb300 import Colony

    wl = aco_synth.WORKLOADS["lbest200k"]
    p = dict(wl["params"])
    xy = aco_synth.make("lbest200k")
    col = Colony(xy, **p)
    cand = col.build_candidates(return_lists=True).cpu().numpy()
    ocand = oracle.knn_sweep(xy, p["k"])  # the oracle's own lists (exact x-sweep)
    yield col, xy, p, cand, ocand
    col.close()


def test_fullsize_candidate_lists(colony200k):
    col, xy, p, cand, ocand = colony200k
    rng = np.random.default_rng(0)
    for i in rng.choice(p["n"], 48, replace=False):
        assert np.array_equal(cand[i], oracle.knn_one(xy, p["k"], int(i))), i
    assert np.array_equal(cand, ocand)


def test_fullsize_iterations(colony200k):
    col, xy, p, cand, ocand = colony200k
    n, m, k, f = p["n"], p["m"], p["k"], p["max_mod_frac"]
    rng = np.random.default_rng(1)
    # initial tours (Algorithm 1, before its iterations)
    tours, lens = col.construct(0, return_tours=True, return_lengths=True)
    T0 = tours.cpu().numpy()
    L0 = lens.cpu().numpy()
    del tours
    sample = rng.choice(m, 12, replace=False)
    for a in sample:
        assert np.array_equal(np.sort(T0[a]), np.arange(n))
    assert np.array_equal(L0[sample], exact_tour_lengths(xy, T0[sample]))
    # eight of the sampled ants rebuilt by the oracle from scratch, one host process each
    built = oracle_pool.initial_tours(xy, ocand, p, sample[:8])
    for a, (t, ln) in built.items():
        assert np.array_equal(t, T0[a]), f"initial tour of ant {a} differs"
        assert ln == L0[a]
    ref = oracle.Oracle(xy, cand=ocand, **p)
    col.update()
    lb, cl, _ = col.state()
    prev_l = cl.cpu().numpy()
    assert np.array_equal(prev_l, L0)
    assert col.stats()["gbest"] == L0.min()
    del T0
    # a PartialACO iteration from the same synthetic l_best population on both sides
    S = aco_synth.snake_tours(xy, m, 7)
    SL = oracle.tour_lengths(xy, S)
    col.set_state(torch.from_numpy(S).cuda())
    lb, cl, _ = col.state()
    assert np.array_equal(cl.cpu().numpy(), SL)
    ref.set_lbest(S, SL)
    prev_l = SL
    for it in range(5, 8):
        tours, lens = col.construct(it, return_tours=True, return_lengths=True)
        if it == 5:
            T = tours.cpu().numpy()
            Ln = lens.cpu().numpy()
            rs = rng.choice(m, 16, replace=False).astype(np.int32)
            ref.construct(it, ants=rs)
            RT = ref.newtours
            RL = ref.newlen
            s, M = ref.segments()
            for a in rs:
                assert 1 <= M[a] <= math.floor(f * n)
                assert np.array_equal(RT[a], T[a]), f"iteration {it}: ant {a} differs from the oracle"
                assert RL[a] == Ln[a]
            del RT, T
        col.update()
        lb, cl, _ = col.state()
        c = cl.cpu().numpy()
        assert np.all(c <= prev_l)
        assert col.stats()["gbest"] == c.min()
        prev_l = c
    L = lb.cpu().numpy()
    chk = rng.choice(m, 16, replace=False)
    for a in chk:
        assert np.array_equal(np.sort(L[a]), np.arange(n))
    assert np.array_equal(prev_l[chk], exact_tour_lengths(xy, L[chk]))
