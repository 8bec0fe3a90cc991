"""Asynchronous l_best sharing: improved partial rebuilds commit inside the construction launch.

The tours then depend on timing, so the oracle has no counterpart.  The tests check what holds
whatever the timing:
  * every l_best is a permutation with its exact length, C_lbest never increases, C_gbest is the
    minimum, and ants commit inside the launch (the improved counter moves before the update);
  * with one ant nothing races: right after the launch, the colony's Eq. 1 probabilities equal
    those of a colony restored from the new l_best (the pheromone moved and the rows reweighted
    exactly);
  * after each update the state is the usual function of the l_best population: a colony
    restored from the same l_best runs the next (synchronous) iteration identically;
  * the mode excludes local search and batches, and runs within 3% of the synchronous colony's
    best tour on a clustered instance.
"""
import numpy as np
import pytest

import aco_synth
from tests.gpu_common import exact_tour_lengths, require_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _colony(xy, **kw):
    from paper_1709_03187_gb300 import Colony

    col = Colony(xy, **kw)
    col.build_candidates()
    return col


def _probs_equal(c1, c2, n, rng, trials=24):
    for _ in range(trials):
        vis = rng.random(n) < rng.random()
        i = int(rng.integers(n))
        vis[i] = True
        p1, e1 = c1.step_probs(i, vis)
        p2, e2 = c2.step_probs(i, vis)
        assert e1 == e2
        assert torch.equal(p1, p2), f"city {i}"


@pytest.mark.parametrize("p_partial", [1.0, 0.5])
def test_invariants_and_commits_inside_the_launch(p_partial):
    """p_partial = 0.5 mixes partial rebuilds (committed in the launch) with full constructions
    (committed by the update step)."""
    require_gpu()
    n, m, k = 2000, 64, 16
    xy = aco_synth.clustered(n, 10, 0.02, 3)
    kw = dict(mode=1, n=n, m=m, k=k, max_mod_frac=0.2, p_partial=p_partial, seed=3)
    col = _colony(xy, **kw)
    col.iterate(0)
    col.set_async_share(True)
    prev = col.state()[1].cpu().numpy()
    inside = 0
    for it in range(1, 9):
        before = col.stats()["improved"]
        col.construct(it)
        inside += col.stats()["improved"] - before  # commits made by the launch itself
        col.update()
        lb, cl, _ = col.state()
        L, C = lb.cpu().numpy(), cl.cpu().numpy()
        for a in range(m):
            assert np.array_equal(np.sort(L[a]), np.arange(n))
        assert np.array_equal(C, exact_tour_lengths(xy, L))
        assert np.all(C <= prev)
        assert col.stats()["gbest"] == C.min()
        prev = C
    assert inside > 0
    # the state after the update is the synchronous function of the l_best population
    ref = _colony(xy, **kw)
    ref.set_state(lb)
    _probs_equal(col, ref, n, np.random.default_rng(0))
    col.set_async_share(False)
    col.iterate(9)
    ref.iterate(9)
    assert np.array_equal(col.state()[0].cpu().numpy(), ref.state()[0].cpu().numpy())
    assert np.array_equal(col.state()[1].cpu().numpy(), ref.state()[1].cpu().numpy())
    col.close()
    ref.close()


@pytest.mark.parametrize("n,k", [(600, 16), (900, 7), (500, 20)])
def test_single_ant_commit_equals_a_restore(n, k):
    """One ant: the in-launch commit (pheromone moved entry by entry, touched rows reweighted,
    half-warp rows for k <= 16, whole-warp rows above) leaves exactly the state of a restore."""
    require_gpu()
    xy = aco_synth.clustered(n, 6, 0.03, n)
    kw = dict(mode=1, n=n, m=1, k=k, max_mod_frac=0.3, seed=5)
    col = _colony(xy, **kw)
    col.iterate(0)
    col.set_async_share(True)
    rng = np.random.default_rng(n)
    commits = 0
    for it in range(1, 80):
        if commits == 3:
            break
        before = col.stats()["improved"]
        col.construct(it)
        if col.stats()["improved"] > before:  # committed in the launch: compare before the update
            commits += 1
            ref = _colony(xy, **kw)
            ref.set_state(col.state()[0])
            _probs_equal(col, ref, n, rng, trials=8)
            ref.close()
        col.update()
    assert commits >= 2
    col.close()


def test_mode_excludes_local_search_and_batches():
    require_gpu()
    from paper_1709_03187_gb300 import AcoError, Batch, Colony

    n = 300
    xy = aco_synth.uniform(n, 2)
    col = _colony(xy, mode=1, n=n, m=8, k=8, seed=1)
    col.set_local_search(0.5, 50)
    with pytest.raises(AcoError):
        col.set_async_share(True)
    col.set_local_search(0.0, 50)
    col.set_async_share(True)
    with pytest.raises(AcoError):
        col.set_local_search(0.5, 50)
    col.construct(0)
    with pytest.raises(AcoError):  # between construct and update
        col.set_async_share(False)
    col.update()
    col.close()
    dense = Colony(xy[:50], mode=0, n=50, m=5, k=0, seed=1)
    with pytest.raises(AcoError):
        dense.set_async_share(True)
    dense.close()
    b = Batch([aco_synth.uniform(60, 1), aco_synth.uniform(80, 2)], m=8, k=6, seed=1)
    from paper_1709_03187_gb300 import _ffi

    with pytest.raises(AcoError):
        _ffi.aco_set_async_share(_ffi.aco_batch_instance(b._h, 0), True)
    b.close()


def test_convergence_close_to_the_synchronous_colony():
    require_gpu()
    n, m, k, iters = 5000, 128, 16, 40
    xy = aco_synth.clustered(n, 25, 0.01, 11)
    kw = dict(mode=1, n=n, m=m, k=k, max_mod_frac=0.1, seed=2)
    best = {}
    for mode in (False, True):
        col = _colony(xy, **kw)
        col.iterate(0)
        col.set_async_share(mode)
        for it in range(1, iters):
            col.iterate(it)
        best[mode] = col.stats()["gbest"]
        col.close()
    assert best[True] <= 1.03 * best[False], best
