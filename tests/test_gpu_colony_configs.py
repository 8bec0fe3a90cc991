"""Whole colonies against the oracle at the sizes of the benchmark configurations (needs a GB300).

  * The 10,000-city configuration (half uniform, half in 20 Gaussian clusters; k = 20, m = 256,
    f = 0.1): k = 20 takes the construction kernel's wide stage (rows of 24 entries) with 32-lane
    scans and the hashed exhausted step.  Every tour, length, l_best and counter bit for bit over
    several iterations.
  * A 2,400-city colony with k = 16 (the staged rows and the hashed exhausted step).
  * In both, the oracle counts exhausted-list picks whose pheromone lies above tau0 (an l_best
    neighbour outside the candidate list, Section 3 pheromone under the Section 6 fallback), and
    the test asserts there were some: the GPU made the same picks, so it took that path too.
  * Asynchronous l_best sharing with one ant: nothing races, so the in-launch commit must leave
    the colony exactly where the synchronous oracle's update leaves it, for ten iterations.
"""
import numpy as np
import pytest

import aco_synth
import oracle
from tests.gpu_common import first_divergence, require_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run_pair(xy, params, iters, cand=None, async_share=False):
    from paper_1709_03187_gb300 import Colony

    require_gpu()
    col = Colony(xy, **params)
    gcand = col.build_candidates(return_lists=True).cpu().numpy()
    ref = oracle.Oracle(xy, cand=cand, **params) if cand is not None else oracle.Oracle(xy, **params)
    assert np.array_equal(gcand, ref.cand)
    for it in range(iters):
        if async_share and it == 1:
            col.set_async_share(True)  # from the first partial rebuild on
        tours, lens = col.construct(it, return_tours=True, return_lengths=True)
        ref.construct(it)
        d = first_divergence(tours.cpu().numpy(), ref.newtours)
        assert d is None, f"iteration {it}: first differing (ant, position) {d}"
        assert np.array_equal(lens.cpu().numpy(), ref.newlen), f"iteration {it}: lengths"
        col.update()
        ref.update()
        lb, cl, _ = col.state()
        assert np.array_equal(lb.cpu().numpy(), ref.lbest), f"iteration {it}: l_best"
        assert np.array_equal(cl.cpu().numpy(), ref.clen), f"iteration {it}: C_lbest"
    st = col.stats()
    c = ref.counters()
    assert st["gbest"] == ref.clen.min()
    assert st["decisions"] == c["decisions"]
    assert st["fallbacks"] == c["fallbacks"]
    col.close()
    return st, c


def test_config_10k_mixed_k20_colony_bit_exact():
    p = dict(aco_synth.WORKLOADS["lbest10k"]["params"])
    xy = aco_synth.make("lbest10k")
    cand = oracle.knn_sweep(xy, p["k"])
    st, c = _run_pair(xy, p, 6, cand=cand)
    assert c["fallbacks"] > 0 and c["boosted"] > 0, c


def test_staged_rows_boosted_exhausted_steps_bit_exact():
    n = 2400
    xy = aco_synth.clustered(n, 12, 0.02, 24)
    p = dict(mode=1, n=n, m=64, k=16, alpha=1.0, beta=2.0, tau0=1.0, max_mod_frac=0.2, p_partial=1.0, seed=24)
    st, c = _run_pair(xy, p, 8)
    assert c["boosted"] > 0, c


# (instances and seeds on which the single ant improves its l_best at least three times in twelve
# iterations, so the in-launch commit is exercised)
@pytest.mark.parametrize("k,xy_seed,seed", [(16, 46, 16), (20, 51, 1), (20, 56, 6)])
def test_async_single_ant_equals_synchronous_oracle(k, xy_seed, seed):
    n = 3000
    xy = aco_synth.clustered(n, 15, 0.02, xy_seed)
    p = dict(mode=1, n=n, m=1, k=k, alpha=1.0, beta=2.0, tau0=1.0, max_mod_frac=0.1, p_partial=1.0, seed=seed)
    st, c = _run_pair(xy, p, 12, async_share=True)
    assert st["improved"] >= 4  # the initial tour and at least three commits inside the launch
