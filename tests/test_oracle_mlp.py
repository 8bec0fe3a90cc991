"""Pins of the learned-proposal oracle (oracle/mlp.py and the edge-score hook of the C oracle).

Each pin comes from outside the oracle's own formulas: central finite differences of the loss
for every gradient entry, hand-built networks and tours with values worked out by hand, closed
forms of the softmax cross-entropy, the bit-level definition of BF16 rounding, and the reduction
of the learned proposal to the plain method when the score equals eta^beta."""
import math

import numpy as np
import pytest

import aco_synth
import oracle
from oracle import mlp

H, IN = mlp.H, mlp.IN


def _rne_bits(x32: np.ndarray) -> np.ndarray:
    """BF16 rounding of float32 values as the bit formula: add 0x7FFF plus the lowest kept bit,
    then clear the low half."""
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def test_bf16_round_ties_and_bits():
    assert mlp.bf16_round(1.0 + 2.0 ** -8) == 1.0                      # tie to the even neighbour
    assert mlp.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6      # tie, odd below, even above
    assert mlp.bf16_round(-(1.0 + 2.0 ** -8 + 2.0 ** -20)) == -(1.0 + 2.0 ** -7)
    assert mlp.bf16_round(3.0) == 3.0
    x = (np.random.default_rng(0).standard_normal(20000) * 10.0).astype(np.float32)
    assert np.array_equal(mlp.bf16_round(x.astype(np.float64)), _rne_bits(x))


def _random_problem(seed, cities=3, k=5, scale=1.0):
    rng = np.random.default_rng(seed)
    X = np.zeros((cities * k, IN))
    X[:, :5] = mlp.bf16_round(rng.uniform(-1.5, 1.5, (cities * k, 5)))
    X[:, 5] = 1.0
    w = aco_synth.mlp_weights(seed).astype(np.float64) * scale * mlp.trainable_mask()
    return X, w


def test_gradients_match_central_differences():
    X, w = _random_problem(3)
    k = 5
    target = np.array([0b00101, 0b10000, 0], np.uint32)  # two targets, one target, none
    _, _, _, a1, a2 = mlp.forward(w, X)
    assert np.abs(a1[:, :H - 1]).min() > 1e-4 and np.abs(a2[:, :H - 1]).min() > 1e-4  # no kink within h
    loss, g, _ = mlp.loss_and_grads(w, X, target, k, scale=0.5)
    h = 1e-6
    fd = np.empty_like(w)
    for e in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        fd[e] = (mlp.loss_and_grads(wp, X, target, k, 0.5)[0] - mlp.loss_and_grads(wm, X, target, k, 0.5)[0]) / (2 * h)
    assert np.all(np.abs(fd - g) <= 1e-6 * (1.0 + np.abs(g))), np.abs(fd - g).max()
    assert np.abs(g).max() > 1e-3
    # the entries training never changes have zero gradient
    assert np.all(g[mlp.trainable_mask() == 0] == 0.0)


def test_hand_built_network():
    W1 = np.zeros((H, IN)); W2 = np.zeros((H, H)); w3 = np.zeros(H)
    W1[0, 0] = 1.0          # h1[0] = relu(x0)
    W1[1, 5] = 0.5          # h1[1] = 0.5 through the bias input
    W2[0, 0] = 2.0; W2[0, 1] = 1.0   # h2[0] = relu(2 h1[0] + h1[1])
    W2[1, H - 1] = -1.0     # h2[1] = relu(-1 * constant unit) = 0
    w3[0] = 3.0; w3[1] = 7.0; w3[H - 1] = 0.25
    w = np.concatenate([W1.ravel(), W2.ravel(), w3])
    X = np.zeros((3, IN)); X[:, 5] = 1.0
    X[:, 0] = [0.75, -1.0, 0.0]
    z = mlp.forward(w, X)[0]
    assert np.array_equal(z, [3.0 * (2 * 0.75 + 0.5) + 0.25, 3.0 * 0.5 + 0.25, 3.0 * 0.5 + 0.25])


def test_cross_entropy_closed_forms():
    k = 4
    w = np.zeros(mlp.N_W1 + mlp.N_W2 + mlp.N_W3)  # every z = 0: softmax is uniform
    X = np.zeros((3 * k, IN)); X[:, 5] = 1.0
    target = np.array([0b0001, 0b1010, 0], np.uint32)
    loss, g, dz = mlp.loss_and_grads(w, X, target, k)
    assert loss == pytest.approx(2 * math.log(k), rel=1e-15)
    dz = dz.reshape(3, k)
    assert np.allclose(dz[0], [0.25 - 1, 0.25, 0.25, 0.25], atol=1e-15)
    assert np.allclose(dz[1], [0.25, 0.25 - 0.5, 0.25, 0.25 - 0.5], atol=1e-15)
    assert np.all(dz[2] == 0.0)
    # non-uniform softmax: the loss of one city with two targets is -(log p_a + log p_b) / 2
    X2, w2 = _random_problem(5, cities=1, k=k)
    z = mlp.forward(w2, X2)[0]
    p = np.exp(z - z.max()) / np.exp(z - z.max()).sum()
    l2 = mlp.loss_and_grads(w2, X2, np.array([0b0110], np.uint32), k)[0]
    assert l2 == pytest.approx(-(math.log(p[1]) + math.log(p[2])) / 2, rel=1e-12)


def test_z_error_bound_covers_bf16_activations():
    """A numpy model of a kernel that rounds h1 and h2 to BF16 and sums in FP32 stays within the
    bound on every row."""
    X, w = _random_problem(7, cities=200, k=8, scale=1.0)
    W1, W2, w3 = (mlp.bf16_round(a) for a in mlp.split(w))
    wb = np.concatenate([W1.ravel(), W2.ravel(), w3])
    f32 = np.float32
    a1 = (X.astype(f32) @ W1.T.astype(f32)).astype(np.float64)
    h1 = mlp.bf16_round(np.maximum(a1, 0)); h1[:, H - 1] = 1
    a2 = (h1.astype(f32) @ W2.T.astype(f32)).astype(np.float64)
    h2 = mlp.bf16_round(np.maximum(a2, 0)); h2[:, H - 1] = 1
    zs = (h2.astype(f32) @ w3.astype(f32)).astype(np.float64)
    z = mlp.forward(wb, X)[0]
    bound = mlp.z_error_bound(wb, X)
    assert np.all(np.abs(zs - z) <= bound)
    assert np.abs(zs - z).max() > 0  # the model does round


def test_features_worked_example():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0], [-3.0, 0.0], [0.0, -4.0]])
    cand = oracle.knn(xy, 4)
    assert list(cand[0]) == [1, 2, 3, 4]
    deg = np.array([2, 4, 6, 8, 32])
    X = mlp.features(xy, cand, deg).reshape(5, 4, IN)
    dbar = 2.5
    assert np.allclose(X[0, :, 0], np.array([1, 2, 3, 4]) / dbar, rtol=1e-15)
    assert np.allclose(X[0, :, 1], [0, 1 / 3, 2 / 3, 1], rtol=1e-15)
    assert np.allclose(X[0, :, 2], np.array([1, 0, -3, 0]) / dbar, rtol=1e-15, atol=0)
    assert np.allclose(X[0, :, 3], np.array([0, 2, 0, -4]) / dbar, rtol=1e-15, atol=0)
    assert np.array_equal(X[0, :, 4], np.array([4, 6, 8, 32]) / 32.0)
    assert np.all(X[..., 5] == 1.0) and np.all(X[..., 6:] == 0.0)


def test_features_invariants():
    xy = aco_synth.clustered(300, 6, 0.02, 9)
    cand = oracle.knn(xy, 10)
    X = mlp.features(xy, cand, np.full(300, 2)).reshape(300, 10, IN)
    assert np.allclose(X[:, :, 0].mean(axis=1), 1.0, rtol=1e-13)
    assert np.allclose(X[:, :, 2] ** 2 + X[:, :, 3] ** 2, X[:, :, 0] ** 2, rtol=1e-12)
    assert np.all(np.diff(X[:, :, 0], axis=1) >= 0)  # candidate lists ascend in distance


def test_degree_worked_example():
    A = np.array([0, 1, 2, 3, 4, 5]); B = np.array([0, 2, 1, 3, 5, 4])
    tours = np.stack([A, B])
    assert np.array_equal(mlp.degree(tours, 1), [2] * 6)
    assert np.array_equal(mlp.degree(tours, 2), [4, 3, 3, 4, 3, 3])
    assert np.array_equal(mlp.degree(np.stack([A, A[::-1]]), 2), [2] * 6)


def test_labels_worked_example():
    tour = np.array([0, 1, 2, 3, 4])
    cand = np.array([[1, 2, 4, 3], [3, 0, 4, 2], [4, 3, 0, 1], [0, 2, 1, 4], [2, 1, 3, 0]])
    assert list(mlp.labels(tour, cand)) == [0b0101, 0b1010, 0b1010, 0b1010, 0b1100]


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([3.0, -0.5, 0.0, 2.0])
    mask = np.array([1, 1, 1, 0])
    w, m1, m2 = mlp.adam_step(np.ones(4), np.zeros(4), np.zeros(4), g, mask, step=1, lr=0.01)
    assert np.allclose(w, [1 - 0.01 * 3 / (3 + 1e-8), 1 + 0.01 * 0.5 / (0.5 + 1e-8), 1.0, 1.0], rtol=1e-15)
    assert m1[3] == 0.0 and m2[3] == 0.0


def test_edge_scores_equal_to_eta_reproduce_the_plain_method():
    xy = aco_synth.clustered(120, 4, 0.05, 2)
    kw = dict(mode=1, n=120, m=8, k=7, max_mod_frac=0.5, seed=3)
    plain = oracle.Oracle(xy, **kw)
    scored = oracle.Oracle(xy, **kw)
    scored.set_edge_scores(plain.etab.copy())
    for it in range(4):
        plain.iterate(it)
        scored.iterate(it)
    assert np.array_equal(plain.lbest, scored.lbest)
    # a constant score leaves only tau; before the first tours tau = tau0 on every edge, so the
    # unvisited candidates are equally likely
    flat = oracle.Oracle(xy, **kw)
    flat.set_edge_scores(np.full((120, 7), 3.5))
    visited = np.zeros(120, np.uint8)
    i = 5
    visited[flat.cand[i, :3]] = 1
    p, ex = flat.step_probs(i, visited)
    assert not ex
    assert np.allclose(p, [0, 0, 0, 0.25, 0.25, 0.25, 0.25], rtol=1e-15, atol=0)
    flat.set_edge_scores(None)
    assert np.array_equal(flat.etab, plain.etab)


def _emulated_kernel_grads(w, X, T, k, scale):
    """A numpy model of the backward kernels' roundings: BF16 h1, h2 in the forward pass, FP32
    softmax, dz * scale in FP32, BF16 dh2 = dz w3 [h2 > 0], BF16 dh1 = (dh2 W2) [h1 > 0], BF16 dz
    for dw3, FP32 sums of the weight-gradient products."""
    f32 = np.float32
    W1, W2, w3 = mlp.split(w)
    a1 = (X.astype(f32) @ W1.T.astype(f32)).astype(np.float64)
    h1 = mlp.bf16_round(np.maximum(a1, 0)); h1[:, H - 1] = 1
    a2 = (h1.astype(f32) @ W2.T.astype(f32)).astype(np.float64)
    h2 = mlp.bf16_round(np.maximum(a2, 0)); h2[:, H - 1] = 1
    z = (h2.astype(f32) @ w3.astype(f32)).reshape(-1, k)
    e = np.exp(z - z.max(axis=1, keepdims=True)).astype(f32)
    p = (e / e.sum(axis=1, keepdims=True, dtype=f32)).astype(f32)
    y = np.zeros_like(p)
    for c, t in enumerate(T):
        r = [b for b in range(k) if (int(t) >> b) & 1]
        y[c, r] = f32(1.0 / len(r)) if r else 0
    live = np.array([int(t) != 0 for t in T])[:, None]
    dz = (np.where(live, p - y, 0).astype(f32) * f32(scale)).reshape(-1).astype(f32)
    dh2 = mlp.bf16_round((dz[:, None] * w3.astype(f32)[None, :]).astype(np.float64) * (h2 > 0))
    dh2[:, H - 1] = 0
    dh1 = mlp.bf16_round((dh2.astype(f32) @ W2.astype(f32)).astype(np.float64) * (h1 > 0))
    dh1[:, H - 1] = 0
    dzb = mlp.bf16_round(dz.astype(np.float64))
    gW2 = dh2.astype(f32).T @ h1.astype(f32)
    gW1 = dh1.astype(f32).T @ X.astype(f32)
    gw3 = dzb.astype(f32) @ h2.astype(f32)
    return np.concatenate([gW1.ravel(), gW2.ravel(), gw3]).astype(np.float64)


def test_grad_error_bound_covers_a_rounding_kernel_entry_by_entry():
    """Against the network with BF16 activations (round_hidden), a numpy model of the kernels'
    roundings stays within the per-entry bound, and the bound is a small fraction of the
    gradients themselves (a wrong entry cannot hide behind it)."""
    X, w = _random_problem(11, cities=300, k=20, scale=1.0)
    W1, W2, w3 = (mlp.bf16_round(a) for a in mlp.split(w))
    wb = np.concatenate([W1.ravel(), W2.ravel(), w3]) * mlp.trainable_mask()
    rng = np.random.default_rng(12)
    T = np.array([sum(1 << int(r) for r in rng.choice(20, rng.integers(0, 3), replace=False)) for _ in range(300)],
                 np.uint32)
    scale = 1.0 / 300
    _, go, _ = mlp.loss_and_grads(wb, X, T, 20, scale=scale, round_hidden=True)
    ge = _emulated_kernel_grads(wb, X, T, 20, scale)
    bound = mlp.grad_error_bound(wb, X, T, 20, scale=scale, round_hidden=True)
    on = mlp.trainable_mask() == 1
    err = np.abs(ge - go)[on]
    assert np.all(err <= 1.25 * bound[on])
    assert err.max() > 0  # the model does round
    assert np.median(bound[on] / (np.abs(go[on]) + 1e-30)) < 0.1


def test_round_hidden_network_pins():
    """round_hidden changes nothing where every activation is already a BF16 value (weights and
    inputs small multiples of powers of two), and otherwise its activations are the exact ones
    rounded to BF16."""
    rng = np.random.default_rng(5)
    X = np.zeros((40, IN))
    X[:, :5] = rng.integers(-1, 2, (40, 5))
    X[:, 5] = 1.0
    W2 = np.zeros((H, H))  # three entries of +-1 per row: |a2| <= 18, an 8-bit integer
    for r in range(H):
        W2[r, rng.choice(H, 3, replace=False)] = rng.choice([-1.0, 1.0], 3)
    w = np.concatenate([rng.integers(-1, 2, H * IN).astype(np.float64), W2.ravel(),
                        rng.integers(-2, 3, H) / 4.0]) * mlp.trainable_mask()
    T = np.array([0b11, 0b100, 0, 0b1000] * 2, np.uint32)
    a = mlp.loss_and_grads(w, X, T, 5)
    b = mlp.loss_and_grads(w, X, T, 5, round_hidden=True)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    Xr, wr = _random_problem(3, cities=20, k=5)
    z0, h10, h20, a10, a20 = mlp.forward(wr, Xr)
    z1, h11, h21, a11, a21 = mlp.forward(wr, Xr, round_hidden=True)
    assert np.array_equal(h11, mlp.bf16_round(h10))
    assert np.array_equal(h21[:, :H - 1], mlp.bf16_round(np.maximum(h11 @ mlp.split(wr)[1].T, 0))[:, :H - 1])
    assert not np.array_equal(z0, z1)
