"""What the trained network gains over the plain heuristic (the plain method is the yardstick).

The network is trained on the GPU from plain runs on small clustered instances (labels: the
candidate ranks of each city's neighbours in the best tour), then scores the candidate edges of
held-out larger clustered instances.  With the same seeds, iterations and parameters, the learned
proposal must end with best tours at least 1% shorter than eta^beta's, and reach the plain run's
final length in at most 75% of its iterations (measured: 3% shorter; 65-70% of the iterations)."""
import numpy as np
import pytest

import aco_synth
from tests.gpu_common import require_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _curve(xy, n, m, k, f, seed, iters, scorer=None):
    from paper_1709_03187_gb300 import Colony

    col = Colony(xy, mode=1, n=n, m=m, k=k, max_mod_frac=f, seed=seed)
    col.build_candidates()
    col.iterate(0)
    if scorer is not None:
        scorer.score(col.handle, n, k, 16, beta=2.0)
    best = [col.stats()["gbest"]]
    for it in range(1, iters):
        col.iterate(it)
        best.append(col.stats()["gbest"])
    col.close()
    return np.array(best)


def test_learned_proposal_beats_the_plain_heuristic():
    require_gpu()
    from paper_1709_03187_gb300 import EdgeScorer
    from paper_1709_03187_gb300.learned import training_data

    xys = [aco_synth.clustered(1000, 5, 0.01, 500 + i) for i in range(150)]
    X, T, _ = training_data(xys, m=32, k=20, iterations=30, seed=3)
    sc = EdgeScorer(aco_synth.mlp_weights(1), max_rows=2048 * 20)
    loss = sc.train(X, T, 20, batch_cities=2048, steps=400, lr=2e-3).cpu().numpy()
    assert loss[-20:].mean() < loss[:20].mean()
    n, iters = 5000, 40
    plain, learned = [], []
    for s in (1, 2):
        xy = aco_synth.clustered(n, 25, 0.01, 7000 + s)
        plain.append(_curve(xy, n, 128, 20, 0.1, s, iters))
        learned.append(_curve(xy, n, 128, 20, 0.1, s, iters, scorer=sc))
    sc.close()
    p_final = np.mean([c[-1] for c in plain])
    l_final = np.mean([c[-1] for c in learned])
    assert l_final < 0.99 * p_final, (p_final, l_final)
    for p, l in zip(plain, learned):
        reach = int(np.argmax(l <= p[-1])) if np.any(l <= p[-1]) else iters
        assert reach + 1 <= 0.75 * iters, (reach, p[-1], l)
