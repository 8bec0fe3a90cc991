"""Batched colonies: every launch schedule -- four launches per iteration replayed as a CUDA graph,
or one persistent cooperative launch with device work queues and grid-wide barriers -- and the
schedule autotuner give exactly what each instance gives alone (and what the oracle gives), bit
for bit.  A persistent launch whose barrier wait runs out reports ACO_ERR_TIMEOUT and leaves the
GPU usable."""
import numpy as np
import pytest

import aco_synth
import oracle
from tests.gpu_common import require_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _instances(count, lo, hi, seed):
    ns = aco_synth.batch_sizes(count, lo, hi, seed)
    return [aco_synth.uniform(int(n), seed * 1000 + i) for i, n in enumerate(ns)]


@pytest.mark.parametrize("tune,schedule", [(False, -1), (True, -1), (False, 8), (False, 9), (False, 10),
                                           (False, 11)])
def test_batch_equals_instances_run_alone(tune, schedule):
    require_gpu()
    from paper_1709_03187_gb300 import Batch, Colony

    xys = _instances(14, 40, 700, 3)
    kw = dict(m=24, k=10, alpha=1.0, beta=2.0, tau0=1.0, max_mod_frac=1.0, seed=11)
    b = Batch(xys, **kw)
    b.set_schedule(schedule)  # 8-11: every iteration in one persistent launch
    b.build_candidates()
    b.run(0, 3)                 # initial tours + 2 iterations (graph replay)
    b.run(3, 6, tune=tune)      # tuning switches schedules over live iterations
    got = b.state()
    best = b.best()
    for i, xy in enumerate(xys):
        n = xy.shape[0]
        col = Colony(xy, mode=1, n=n, m=min(n, 24), k=10, alpha=1.0, beta=2.0, tau0=1.0, max_mod_frac=1.0,
                     seed=11 + i)
        col.build_candidates()
        for it in range(9):
            col.iterate(it)
        lb, cl, _ = col.state()
        assert np.array_equal(got[i][0], lb.cpu().numpy()), f"instance {i} (n={n}) l_best differs"
        assert np.array_equal(got[i][1], cl.cpu().numpy())
        assert best[i] == cl.min().item()
        col.close()
    (sc, w, mb, pull), ms = b.schedule()
    assert w in (1, 2, 4, 8) and mb in (2, 4, 8, 16, 24, 32)
    if schedule >= 0:
        assert sc == schedule and pull >= 1
    if tune:
        assert np.all(ms[:6] > 0)  # six tuned iterations in the second call
    b.close()


def test_persistent_batch_matches_oracle_with_mixed_k16_rows():
    """k = 16: the staged candidate rows inside the persistent launch."""
    require_gpu()
    from paper_1709_03187_gb300 import Batch

    xys = [aco_synth.clustered(300, 5, 0.03, 21), aco_synth.uniform(77, 22), aco_synth.clustered(520, 6, 0.02, 23)]
    b = Batch(xys, m=20, k=16, max_mod_frac=0.4, seed=9)
    b.set_schedule(8)
    b.build_candidates()
    b.run(0, 7)
    got = b.state()
    for i, xy in enumerate(xys):
        n = xy.shape[0]
        ref = oracle.Oracle(xy, mode=1, n=n, m=min(n, 20), k=16, max_mod_frac=0.4, seed=9 + i)
        for it in range(7):
            ref.iterate(it)
        assert np.array_equal(got[i][0], ref.lbest), f"instance {i}"
        assert np.array_equal(got[i][1], ref.clen)
    b.close()


def test_persistent_barrier_wait_limit_gives_timeout():
    """A wait limit of zero: a block that is not the last to arrive gives up at once, every block
    leaves, the host reports ACO_ERR_TIMEOUT, the batch refuses to run on, and the GPU is fine."""
    require_gpu()
    from paper_1709_03187_gb300 import AcoError, Batch

    xys = _instances(6, 60, 400, 7)
    b = Batch(xys, m=16, k=8, max_mod_frac=1.0, seed=3)
    b.set_schedule(8)
    b.set_wait_limit(0.0)
    b.build_candidates()
    b.run(0, 3)
    with pytest.raises(AcoError) as e:
        b.best()
    assert e.value.status == 5  # ACO_ERR_TIMEOUT
    with pytest.raises(AcoError) as e:
        b.run(3, 1)
    assert e.value.status == 4  # ACO_ERR_STATE
    b.close()
    # the device is healthy: a new batch with the default limit runs and matches itself alone
    b2 = Batch(xys, m=16, k=8, max_mod_frac=1.0, seed=3)
    b2.set_schedule(8)
    b2.build_candidates()
    b2.run(0, 3)
    assert np.all(np.isfinite(b2.best()))
    b2.close()


def test_batch_matches_oracle():
    require_gpu()
    from paper_1709_03187_gb300 import Batch

    xys = [aco_synth.clustered(90, 3, 0.05, 1), aco_synth.uniform(47, 2), aco_synth.clustered(130, 4, 0.03, 3)]
    b = Batch(xys, m=12, k=7, max_mod_frac=0.5, seed=5)
    b.build_candidates()
    b.run(0, 6, tune=True)
    got = b.state()
    for i, xy in enumerate(xys):
        n = xy.shape[0]
        ref = oracle.Oracle(xy, mode=1, n=n, m=min(n, 12), k=7, max_mod_frac=0.5, seed=5 + i)
        for it in range(6):
            ref.iterate(it)
        assert np.array_equal(got[i][0], ref.lbest)
        assert np.array_equal(got[i][1], ref.clen)
    b.close()
