"""Windowed 2-opt local search on the GPU against the oracle, bit for bit (§8(f) F1)."""
import numpy as np
import pytest

import aco_synth
import oracle
from tests.gpu_common import require_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,m,k,f,p,W,seed", [
    (1500, 16, 12, 0.3, 0.3, 40, 1),   # about 19 blocks per pass and a ragged last block
    (200, 12, 8, 1.0, 1.0, 300, 2),    # one block covering the tour; the 8-ant cap binds
    (2600, 8, 16, 0.05, 0.5, 500, 3),  # the paper's window, partial rebuilds of 130 cities
    (1200, 8, 20, 0.2, 0.5, 100, 4),   # k = 20: construction on the 24-entry stage
])
def test_local_search_matches_oracle(n, m, k, f, p, W, seed):
    require_gpu()
    from paper_1709_03187_gb300 import Colony

    xy = aco_synth.clustered(n, 9, 0.02, 100 + seed)
    kw = dict(mode=1, n=n, m=m, k=k, max_mod_frac=f, seed=seed)
    col = Colony(xy, **kw)
    cand = col.build_candidates(return_lists=True).cpu().numpy()
    ocand = oracle.knn(xy, k)  # the oracle's own lists
    assert np.array_equal(cand, ocand)
    ref = oracle.Oracle(xy, cand=ocand, **kw)
    col.set_local_search(p, W)
    ref.set_local_search(p, W)
    for it in range(5):
        tours, lens = col.construct(it, return_tours=True, return_lengths=True)
        ref.construct(it)
        assert np.array_equal(tours.cpu().numpy(), ref.newtours), f"iteration {it}: new tours"
        assert np.array_equal(lens.cpu().numpy(), ref.newlen)
        col.update()
        ref.update()
        lb, cl, _ = col.state()
        assert np.array_equal(lb.cpu().numpy(), ref.lbest), f"iteration {it}: l_best"
        assert np.array_equal(cl.cpu().numpy(), ref.clen)
    st = col.stats()
    assert st["ls_moves"] == ref.ls_moves and st["ls_moves"] > 0
    col.close()


def test_local_search_arguments():
    require_gpu()
    from paper_1709_03187_gb300 import AcoError, Colony

    col = Colony(aco_synth.uniform(100, 1), mode=1, n=100, m=4, k=8)
    col.build_candidates()
    for p, W in [(1.5, 10), (-0.1, 10), (0.5, 1), (0.5, 5000)]:
        with pytest.raises(AcoError) as e:
            col.set_local_search(p, W)
        assert e.value.status == 1
    col.set_local_search(0.0, 10)  # off: nothing allocated, nothing run
    col.iterate(0)
    assert col.stats()["ls_moves"] == 0
    col.close()
