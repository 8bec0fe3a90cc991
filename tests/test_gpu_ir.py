"""Independent Roulette (selection = 1) on the GPU against the oracle, bit for bit."""
import numpy as np
import pytest

import aco_synth
import oracle
from tests.gpu_common import require_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,m,k,f,seed", [(300, 16, 8, 0.5, 3), (2000, 24, 16, 0.2, 5), (777, 8, 10, 1.0, 9),
                                          (1500, 16, 20, 0.3, 11)])  # k = 20: the 24-entry stage
def test_ir_colony_matches_oracle(n, m, k, f, seed):
    require_gpu()
    from paper_1709_03187_gb300 import Colony

    xy = aco_synth.clustered(n, 7, 0.03, seed)
    kw = dict(mode=1, n=n, m=m, k=k, max_mod_frac=f, seed=seed, selection=1)
    col = Colony(xy, **kw)
    cand = col.build_candidates(return_lists=True).cpu().numpy()
    ocand = oracle.knn(xy, k)  # the oracle's own lists
    assert np.array_equal(cand, ocand)
    ref = oracle.Oracle(xy, cand=ocand, **kw)
    for it in range(5):
        col.iterate(it)
        ref.iterate(it)
        lb, cl, _ = col.state()
        assert np.array_equal(lb.cpu().numpy(), ref.lbest), f"iteration {it}"
        assert np.array_equal(cl.cpu().numpy(), ref.clen)
    st = col.stats()
    c = ref.counters()
    assert st["decisions"] == c["decisions"] and st["fallbacks"] == c["fallbacks"]
    col.close()


def test_ir_differs_from_the_wheel_and_is_rejected_in_dense_mode():
    require_gpu()
    from paper_1709_03187_gb300 import AcoError, Colony

    xy = aco_synth.uniform(200, 4)
    tours = []
    for sel in (0, 1):
        col = Colony(xy, mode=1, n=200, m=8, k=8, seed=2, selection=sel)
        col.build_candidates()
        col.iterate(0)
        col.iterate(1)
        tours.append(col.state()[0].cpu().numpy())
        col.close()
    assert not np.array_equal(tours[0], tours[1])
    with pytest.raises(AcoError):
        Colony(aco_synth.uniform(50, 1), mode=0, n=50, m=4, selection=1)


def test_f_schedule_and_p_partial_match_oracle():
    """F3: the modification limit grows between iterations (and p_partial changes) exactly as
    in the oracle."""
    require_gpu()
    from paper_1709_03187_gb300 import AcoError, Colony, linear_f_schedule

    n, m, k = 900, 16, 12
    xy = aco_synth.clustered(n, 9, 0.02, 21)
    kw = dict(mode=1, n=n, m=m, k=k, max_mod_frac=0.4, seed=8)
    col = Colony(xy, **kw)
    cand = col.build_candidates(return_lists=True).cpu().numpy()
    ocand = oracle.knn(xy, k)  # the oracle's own lists
    assert np.array_equal(cand, ocand)
    ref = oracle.Oracle(xy, cand=ocand, **kw)
    sched = linear_f_schedule(0.01, 0.4, 5)
    for it in range(8):
        col.set_max_mod_frac(sched(it))
        ref.set_max_mod_frac(sched(it))
        if it == 6:
            col.set_p_partial(0.5)
            ref.set_p_partial(0.5)
        col.iterate(it)
        ref.iterate(it)
        lb, cl, _ = col.state()
        assert np.array_equal(lb.cpu().numpy(), ref.lbest), f"iteration {it}"
        assert np.array_equal(cl.cpu().numpy(), ref.clen)
    with pytest.raises(AcoError) as e:
        col.set_max_mod_frac(0.41)  # above the creation value
    assert e.value.status == 1
    col.construct(8)
    with pytest.raises(AcoError) as e:
        col.set_max_mod_frac(0.1)  # between construct and update
    assert e.value.status == 4
    col.update()
    col.close()
