"""Batched colonies: one launch per step over many instances of uneven size, CUDA-graph replay
and the schedule autotuner give exactly what each instance gives alone (and what the oracle
gives), bit for bit."""
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


@pytest.mark.parametrize("tune", [False, True])
def test_batch_equals_instances_run_alone(tune):
    require_gpu()
    from paper_1709_03187_gb300 import Batch, Colony

    xys = _instances(14, 40, 700, 3)
    kw = dict(m=24, k=10, alpha=1.0, beta=2.0, tau0=1.0, max_mod_frac=1.0, seed=11)
    b = Batch(xys, **kw)
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
    (w, mb), ms = b.schedule()
    assert w in (1, 2, 4) and mb in (4, 8, 16, 24, 32)
    if tune:
        assert np.all(ms[:6] > 0)  # six tuned iterations in the second call
    b.close()


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
