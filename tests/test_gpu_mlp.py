"""Learned edge proposal on the GPU against the FP64 oracle (oracle/mlp.py, oracle edge scores).

Network outputs are compared with the oracle's FP64 network on the same BF16 weights and inputs
within the a-priori bound of BF16 hidden activations; every gradient entry within the a-priori
bound of the kernels' roundings against the network with BF16 activations; the features within
one BF16 step; degree counts, labels and every tour built
with learned scores bit for bit."""
import numpy as np
import pytest

import aco_synth
import oracle
from oracle import mlp
from tests.gpu_common import require_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H, IN = mlp.H, mlp.IN


def _features(rows, seed):
    X = np.zeros((rows, IN), np.float32)
    X[:, :5] = aco_synth.bf16_values((rows, 5), seed, -1.5, 1.5)
    X[:, 5] = 1.0
    return X


def _to_dev_bf16(X):
    return torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda().to(torch.bfloat16)


def _oracle_weights(w32):
    return mlp.bf16_round(w32.astype(np.float64) * mlp.trainable_mask())


@pytest.mark.parametrize("rows", [1, 17, 3007])
def test_forward_within_bf16_bound(rows):
    require_gpu()
    from paper_1709_03187_gb300 import EdgeScorer

    w = aco_synth.mlp_weights(21)
    X = _features(rows, 4)
    sc = EdgeScorer(w, max_rows=1 << 12)
    z, s = sc.forward(_to_dev_bf16(X), z=True, score=True)
    z, s = z.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64)
    s2 = sc.forward(_to_dev_bf16(X), z=False, score=True, beta=2.0).cpu().numpy().astype(np.float64)
    wo = _oracle_weights(w)
    zo = mlp.forward(wo, X)[0]
    bound = mlp.z_error_bound(wo, X)
    assert np.all(np.abs(z - zo) <= 1.05 * bound + 1e-6), np.max(np.abs(z - zo) - bound)
    assert np.all(np.abs(np.log(s) - np.clip(zo, -60, 60)) <= 1.05 * bound + 2e-6)
    assert np.all(np.abs(np.log(s2) - np.clip(2 * zo, -60, 60)) <= 2 * 1.05 * bound + 4e-6)
    sc.close()


def _targets(cities, k, seed):
    rng = np.random.default_rng(seed)
    t = np.zeros(cities, np.int64)
    for c in range(cities):
        nb = rng.integers(0, 3)  # 0, 1 or 2 labelled ranks
        for r in rng.choice(k, nb, replace=False):
            t[c] |= 1 << int(r)
    return t.astype(np.int32)


def test_backward_matches_oracle_gradients():
    require_gpu()
    from paper_1709_03187_gb300 import EdgeScorer

    cities, k = 700, 20
    w = aco_synth.mlp_weights(5)
    X = _features(cities * k, 8)
    T = _targets(cities, k, 9)
    sc = EdgeScorer(w, max_rows=cities * k)
    g, loss = sc.backward(_to_dev_bf16(X), torch.from_numpy(T).cuda(), k, scale=1.0 / cities)
    g = g.cpu().numpy().astype(np.float64)
    # the network with BF16 activations, and per entry the a-priori bound of the kernels' roundings
    wo, To = _oracle_weights(w), T.astype(np.uint32)
    lo, go, _ = mlp.loss_and_grads(wo, X, To, k, scale=1.0 / cities, round_hidden=True)
    bound = 1.25 * mlp.grad_error_bound(wo, X, To, k, scale=1.0 / cities, round_hidden=True)
    assert loss.item() == pytest.approx(lo, rel=1e-3)
    on = mlp.trainable_mask() == 1
    err = np.abs(g - go)
    bad = np.nonzero(on & (err > bound))[0]
    assert bad.size == 0, f"{bad.size} entries off bound, first {bad[0]}: gpu {g[bad[0]]} oracle {go[bad[0]]}"
    assert np.all(g[~on] == 0.0)
    sc.close()


def test_adam_steps_match_oracle():
    require_gpu()
    from paper_1709_03187_gb300 import EdgeScorer

    w = aco_synth.mlp_weights(2)
    sc = EdgeScorer(w, max_rows=64)
    mask = mlp.trainable_mask()
    wo, m1, m2 = w.astype(np.float64) * mask, np.zeros(w.size), np.zeros(w.size)
    for step in range(1, 4):
        grad = aco_synth.bf16_values(w.size, 30 + step, -0.1, 0.1)
        sc.adam(torch.from_numpy(grad).cuda(), 1e-2)
        wo, m1, m2 = mlp.adam_step(wo, m1, m2, grad, mask, step, 1e-2)
    got = sc.weights().astype(np.float64)
    assert np.allclose(got, wo, rtol=1e-5, atol=1e-7)
    sc.close()


def test_training_is_deterministic_and_lowers_the_loss():
    require_gpu()
    from paper_1709_03187_gb300 import EdgeScorer

    cities, k = 3000, 16
    X = _to_dev_bf16(_features(cities * k, 1))
    # labels that depend on the features: the two rows with the smallest x0
    x0 = X.float().cpu().numpy()[:, 0].reshape(cities, k)
    T = np.zeros(cities, np.int64)
    for c in range(cities):
        for r in np.argsort(x0[c], kind="stable")[:2]:
            T[c] |= 1 << int(r)
    T = torch.from_numpy(T.astype(np.int32)).cuda()
    runs = []
    for _ in range(2):
        sc = EdgeScorer(aco_synth.mlp_weights(3), max_rows=500 * k)
        loss = sc.train(X, T, k, batch_cities=500, steps=120, lr=3e-3).cpu().numpy()
        runs.append((sc.weights(), loss))
        sc.close()
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    loss = runs[0][1]
    assert loss[-12:].mean() < 0.7 * loss[:12].mean()


def test_features_degree_and_labels_match_oracle():
    require_gpu()
    from paper_1709_03187_gb300 import Colony, EdgeScorer

    n, m, k = 500, 20, 12
    xy = aco_synth.clustered(n, 8, 0.03, 4)
    col = Colony(xy, mode=1, n=n, m=m, k=k, max_mod_frac=0.5, seed=2)
    gcand = col.build_candidates(return_lists=True).cpu().numpy()
    cand = oracle.knn(xy, k)  # the oracle's own lists feed its features
    assert np.array_equal(gcand, cand)
    tours = aco_synth.permutations(m, n, 6)
    col.set_state(torch.from_numpy(tours).cuda())
    lens = oracle.tour_lengths(xy, tours)
    for D in (16, 5, 1):
        X = EdgeScorer.features(col.handle, n, k, degree_ants=D).float().cpu().numpy().astype(np.float64)
        Xo = mlp.bf16_round(mlp.features(xy, cand, mlp.degree(tours, D)))
        exact = [1, 4, 5] + list(range(6, IN))
        assert np.array_equal(X[:, exact], Xo[:, exact]), f"D={D}"
        near = [0, 2, 3]
        assert np.all(np.abs(X[:, near] - Xo[:, near]) <= 2.0 ** -7 * np.abs(Xo[:, near]) + 1e-30)
    T = EdgeScorer.labels(col.handle, n).cpu().numpy().astype(np.uint32)
    best = int(np.argmin(lens))  # ties: the lowest ant index
    assert np.array_equal(T, mlp.labels(tours[best], cand))
    col.close()


@pytest.mark.parametrize("when", [0, 2])
def test_tours_with_learned_scores_match_oracle(when):
    require_gpu()
    from paper_1709_03187_gb300 import Colony, aco_set_edge_scores

    n, m, k = 400, 16, 10
    xy = aco_synth.clustered(n, 6, 0.04, 12)
    kw = dict(mode=1, n=n, m=m, k=k, max_mod_frac=0.5, seed=7)
    col = Colony(xy, **kw)
    col.build_candidates()
    ref = oracle.Oracle(xy, **kw)
    scores = aco_synth.edge_scores(n, k, 13)
    for it in range(6):
        if it == when:
            aco_set_edge_scores(col.handle, torch.from_numpy(scores).cuda())
            ref.set_edge_scores(scores.astype(np.float64))
        if it == 4:  # back to the plain heuristic
            aco_set_edge_scores(col.handle, None)
            ref.set_edge_scores(None)
        col.iterate(it)
        ref.iterate(it)
        lb, cl, _ = col.state()
        assert np.array_equal(lb.cpu().numpy(), ref.lbest), f"iteration {it}"
        assert np.array_equal(cl.cpu().numpy(), ref.clen)
    col.close()


def test_bad_scores_are_rejected_and_leave_the_scores_in_use():
    require_gpu()
    from paper_1709_03187_gb300 import AcoError, Colony, aco_set_edge_scores

    n, m, k = 200, 8, 8
    xy = aco_synth.uniform(n, 3)
    kw = dict(mode=1, n=n, m=m, k=k, seed=1)
    col = Colony(xy, **kw)
    col.build_candidates()
    ref = oracle.Oracle(xy, **kw)
    good = aco_synth.edge_scores(n, k, 4)
    aco_set_edge_scores(col.handle, torch.from_numpy(good).cuda())
    ref.set_edge_scores(good.astype(np.float64))
    for bad_value in (0.0, -1.0, float("nan"), float("inf")):
        bad = good.copy()
        bad[17, 3] = bad_value
        with pytest.raises(AcoError) as e:
            aco_set_edge_scores(col.handle, torch.from_numpy(bad).cuda())
        assert e.value.status == 1
    for it in range(3):
        col.iterate(it)
        ref.iterate(it)
    assert np.array_equal(col.state()[0].cpu().numpy(), ref.lbest)
    col.close()


def test_forward_many_tiles_per_cta_and_ragged_tail():
    """Enough rows that every CTA of the tensor-core forward loops over several 128-row tiles, and
    a last tile of 77 rows: every row within the a-priori bound against the FP64 network."""
    require_gpu()
    from paper_1709_03187_gb300 import EdgeScorer

    rows = 3 * 456 * 128 + 77
    w = aco_synth.mlp_weights(33)
    X = _features(rows, 12)
    sc = EdgeScorer(w, max_rows=1 << 12)
    z = sc.forward(_to_dev_bf16(X), z=True, score=False).cpu().numpy().astype(np.float64)
    wo = _oracle_weights(w)
    zo = mlp.forward(wo, X)[0]
    bound = mlp.z_error_bound(wo, X)
    assert np.all(np.abs(z - zo) <= 1.05 * bound + 1e-6), np.max(np.abs(z - zo) - bound)
    sc.close()


def test_misaligned_features_are_refused():
    """The kernels read features in 4-byte words: a feature pointer at an odd BF16 offset is
    refused with ACO_ERR_INVALID_ARG before anything is enqueued."""
    require_gpu()
    from paper_1709_03187_gb300 import AcoError, EdgeScorer, _ffi

    w = aco_synth.mlp_weights(3)
    sc = EdgeScorer(w, max_rows=64)
    flat = _to_dev_bf16(_features(33, 2)).reshape(-1)
    odd = flat[1:1 + 32 * IN]  # starts 2 bytes into the buffer
    z = torch.empty(32, dtype=torch.float32, device="cuda")
    with pytest.raises(AcoError) as e:
        _ffi.aco_mlp_forward(sc._h, odd, 32, z, None, 1.0)
    assert e.value.status == 1
    zz = sc.forward(flat[: 32 * IN].reshape(32, IN), z=True)  # the aligned view still works
    assert bool(torch.isfinite(zz).all())
    sc.close()
