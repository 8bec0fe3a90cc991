"""FP64 oracle of the learned edge proposal (test infrastructure only).

Plain numpy definitions of what the learned-proposal kernels compute, for the parity tests: the
per-candidate-edge features, the degree-in-best-tours count, the best-tour labels, the 3-layer
MLP forward pass, the softmax cross-entropy over each city's candidate edges and its gradients,
and one Adam step.  The network runs in FP64 on BF16-valued weights and inputs; it does not round
its hidden activations (the kernels do, and ``z_error_bound`` states by how much that may move
the output).  Only ``tests/`` and the benchmark's CPU-baseline leg may import this module.

The learned proposal extends the method (the score stands in for eta^beta of Eq. 1 on candidate
edges, Section 3's candidate lists); the paper gives no network, so every definition here is the
reading written down with the kernels:

  features of candidate edge (i, r), j = cand[i][r], dbar_i = mean_r d(i, cand[i][r]):
    x0 = d_ij / dbar_i, x1 = r / (k - 1), x2 = (x_j - x_i) / dbar_i, x3 = (y_j - y_i) / dbar_i,
    x4 = deg_j / 32, x5 = 1 (bias input), x6..x15 = 0
  deg_j = number of distinct neighbours of j over the l_best tours of ants 0 .. D-1
  network: h1 = relu(W1 x), h1[63] = 1;  h2 = relu(W2 h1), h2[63] = 1;  z = w3 . h2
  loss of city i: -sum_r y_ir log softmax_r(z_i.), y_ir = 1/t_i on the t_i candidate ranks that
    are neighbours of i in the best tour (cities with t_i = 0 are left out)
"""
from __future__ import annotations

import numpy as np

IN, H = 16, 64
N_W1, N_W2, N_W3 = H * IN, H * H, H


def bf16_round(x) -> np.ndarray:
    """Round FP64 values to the nearest BF16 value (8 significant bits), ties to even.

    Written from the format's definition: x = m * 2^e with m in [0.5, 1); keep m * 2^8 rounded to
    an integer (np.rint rounds halves to even)."""
    x = np.asarray(x, np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0), e - 8)


def trainable_mask() -> np.ndarray:
    """1 for every weight that training may change, over the flat (W1, W2, w3) vector.

    Rows 63 of W1 and W2 feed the constant units and W1's columns 6..15 meet zero inputs."""
    m1 = np.zeros((H, IN), np.uint8)
    m1[: H - 1, :6] = 1
    m2 = np.ones((H, H), np.uint8)
    m2[H - 1, :] = 0
    m3 = np.ones(H, np.uint8)
    return np.concatenate([m1.ravel(), m2.ravel(), m3])


def split(wflat):
    w = np.asarray(wflat, np.float64)
    return w[:N_W1].reshape(H, IN), w[N_W1:N_W1 + N_W2].reshape(H, H), w[N_W1 + N_W2:]


def degree(lbest: np.ndarray, ants: int) -> np.ndarray:
    """deg_j: distinct neighbours of every city over the first `ants` tours (brute force)."""
    n = lbest.shape[1]
    nbrs = [set() for _ in range(n)]
    for a in range(min(ants, lbest.shape[0])):
        t = lbest[a]
        for p in range(n):
            c, s = int(t[p]), int(t[(p + 1) % n])
            nbrs[c].add(s)
            nbrs[s].add(c)
    return np.array([len(s) for s in nbrs], np.int64)


def features(xy: np.ndarray, cand: np.ndarray, deg: np.ndarray) -> np.ndarray:
    """FP64 features [n*k][16] of the candidate edges in (city, rank) order."""
    n, k = cand.shape
    X = np.zeros((n, k, IN), np.float64)
    for i in range(n):
        dx = xy[cand[i], 0] - xy[i, 0]
        dy = xy[cand[i], 1] - xy[i, 1]
        d = np.sqrt(dx * dx + dy * dy)
        dbar = d.mean()
        X[i, :, 0] = d / dbar
        X[i, :, 1] = np.arange(k) / (k - 1) if k > 1 else 0.0
        X[i, :, 2] = dx / dbar
        X[i, :, 3] = dy / dbar
        X[i, :, 4] = deg[cand[i]] / 32.0
        X[i, :, 5] = 1.0
    return X.reshape(n * k, IN)


def labels(tour: np.ndarray, cand: np.ndarray) -> np.ndarray:
    """Per city the bitmask of candidate ranks r whose city is a neighbour of i in `tour`."""
    n, k = cand.shape
    succ = np.empty(n, np.int64)
    pred = np.empty(n, np.int64)
    succ[tour] = np.roll(tour, -1)
    pred[tour] = np.roll(tour, 1)
    out = np.zeros(n, np.uint32)
    for i in range(n):
        for r in range(k):
            if cand[i, r] == succ[i] or cand[i, r] == pred[i]:
                out[i] |= np.uint32(1 << r)
    return out


def forward(wflat, X, round_hidden: bool = False):
    """z, h1, h2 and the pre-activations a1, a2 of every row, in FP64.

    round_hidden: round h1 and h2 to BF16 after their FP64 sums, as the network of the learned
    proposal is defined (BF16 weights and activations); the default keeps them exact (the
    differentiable network the finite-difference pins check)."""
    W1, W2, w3 = split(wflat)
    X = np.asarray(X, np.float64)
    a1 = X @ W1.T
    h1 = np.maximum(a1, 0.0)
    if round_hidden:
        h1 = bf16_round(h1)
    h1[:, H - 1] = 1.0
    a2 = h1 @ W2.T
    h2 = np.maximum(a2, 0.0)
    if round_hidden:
        h2 = bf16_round(h2)
    h2[:, H - 1] = 1.0
    z = h2 @ w3
    return z, h1, h2, a1, a2


def z_error_bound(wflat, X) -> np.ndarray:
    """Per row, how far a kernel that rounds h1 and h2 to BF16 (unit roundoff 2^-8) and sums in
    FP32 (at most 64 terms, gamma = 64 * 2^-24) may move z from the FP64 value: the rounding
    errors propagated through |W2| and |w3| to first order."""
    W1, W2, w3 = split(wflat)
    X = np.asarray(X, np.float64)
    u, g = 2.0 ** -8, 64 * 2.0 ** -24
    _, h1, h2, a1, a2 = forward(wflat, X)
    S1 = np.abs(X) @ np.abs(W1).T
    e1 = u * np.abs(h1) + (1 + u) * g * S1
    e1[:, H - 1] = 0.0
    S2 = np.abs(h1) @ np.abs(W2).T
    e2 = e1 @ np.abs(W2).T + g * S2 + u * (np.abs(a2) + e1 @ np.abs(W2).T + g * S2)
    e2[:, H - 1] = 0.0
    return e2 @ np.abs(w3) + g * (np.abs(h2) @ np.abs(w3))


def grad_error_bound(wflat, X, target, k: int, scale: float = 1.0, rows_per_block: int = 256,
                     round_hidden: bool = False) -> np.ndarray:
    """Per weight entry, how far the gradient of a kernel may lie from ``loss_and_grads``' FP64
    gradient when it rounds h1 and h2 to BF16 in the forward pass, computes the softmax in FP32,
    rounds dh2 = dz w3, dh1 = dh2 W2 and dz itself to BF16 for the weight-gradient products, and
    sums those products in FP32 in blocks of `rows_per_block` rows (then the blocks in order).

    First-order propagation of every rounding, as in ``z_error_bound``: the z error moves the
    softmax by at most p_r (e_r + sum_s p_s e_s); a mask [a > 0] may differ where |a| is within
    its own error, and there the whole product counts as error; an FP32 sum of K terms errs by
    at most K 2^-24 times the sum of their magnitudes.  Returned over the flat (W1, W2, w3) vector;
    the caller adds a factor for the second-order terms.

    round_hidden: the bound against ``loss_and_grads(..., round_hidden=True)``, whose h1 and h2 are
    already rounded to BF16.  A kernel's activation then differs from the oracle's only where its
    FP32 sum and the FP64 one round to different BF16 values: by at most
    bf16(relu(a + e)) - bf16(relu(a - e)) for a sum error e (zero away from rounding boundaries)."""
    W1, W2, w3 = split(wflat)
    X = np.asarray(X, np.float64)
    u, g = 2.0 ** -8, 64 * 2.0 ** -24
    aW1, aW2, aw3, aX = np.abs(W1), np.abs(W2), np.abs(w3), np.abs(X)
    z, h1, h2, a1, a2 = forward(wflat, X, round_hidden)
    # forward errors (pre-activation a, activation h after rounding, output z)
    S1 = aX @ aW1.T
    if round_hidden:
        gr = g + 2.0 ** -50  # the oracle's own FP64 sums decide its roundings too
        e1_pre = gr * S1
        e1 = bf16_round(np.maximum(a1 + e1_pre, 0.0)) - bf16_round(np.maximum(a1 - e1_pre, 0.0))
        e1[:, H - 1] = 0.0
        S2 = np.abs(h1) @ aW2.T
        e2_pre = e1 @ aW2.T + gr * S2
        e2 = bf16_round(np.maximum(a2 + e2_pre, 0.0)) - bf16_round(np.maximum(a2 - e2_pre, 0.0))
        e2[:, H - 1] = 0.0
        ez = e2 @ aw3 + gr * (np.abs(h2) @ aw3)
    else:
        e1_pre = g * S1
        e1 = u * np.abs(h1) + (1 + u) * e1_pre
        e1[:, H - 1] = 0.0
        S2 = np.abs(h1) @ aW2.T
        e2_pre = e1 @ aW2.T + g * S2
        e2 = e2_pre + u * (np.abs(a2) + e2_pre)
        e2[:, H - 1] = 0.0
        ez = e2 @ aw3 + g * (np.abs(h2) @ aw3)
    # softmax per city (FP32 exp and division: 2^-18 relative, generous)
    cities = len(target)
    zc = z.reshape(cities, k)
    live = np.array([int(t) != 0 for t in target])
    p = np.exp(zc - zc.max(axis=1, keepdims=True))
    p /= p.sum(axis=1, keepdims=True)
    ezc = ez.reshape(cities, k)
    ep = p * (ezc + (p * ezc).sum(axis=1, keepdims=True)) + 2.0 ** -18 * p
    _, _, dz = loss_and_grads(wflat, X, target, k, 1.0, round_hidden)
    D = np.abs(scale * dz)
    eD = (np.abs(scale) * np.where(live[:, None], ep, 0.0)).reshape(-1) + 2.0 ** -24 * D
    # dh2 = D w3 [a2 > 0], rounded to BF16
    P2 = np.outer(D, aw3)
    on2 = a2 > 0
    flip2 = np.abs(a2) <= e2_pre
    edh2 = on2 * ((1 + u) * np.outer(eD, aw3) + (u + 2.0 ** -24) * P2) + flip2 * P2
    edh2[:, H - 1] = 0.0
    dh2 = P2 * on2
    dh2[:, H - 1] = 0.0
    # dh1 = (dh2 W2) [a1 > 0], rounded to BF16
    T1 = dh2 @ aW2
    E1 = edh2 @ aW2
    on1 = a1 > 0
    flip1 = np.abs(a1) <= e1_pre
    edh1 = on1 * ((1 + u) * (E1 + g * T1) + u * T1) + flip1 * (T1 + E1)
    edh1[:, H - 1] = 0.0
    dh1 = T1 * on1
    dh1[:, H - 1] = 0.0
    # weight gradients: FP32 sums over rows, block partials then the blocks in order
    # (tensor-core accumulation may truncate rather than round: twice the rounding bound)
    R = X.shape[0]
    gam = 2 * (rows_per_block + -(-R // rows_per_block) + 2) * 2.0 ** -24
    eD16 = eD + u * (D + eD)  # dz rounded to BF16 for dw3
    gW2 = edh2.T @ np.abs(h1) + dh2.T @ e1 + edh2.T @ e1 + gam * (dh2.T @ np.abs(h1))
    gW1 = edh1.T @ aX + gam * (dh1.T @ aX)
    gw3 = eD16 @ np.abs(h2) + D @ e2 + eD16 @ e2 + gam * (D @ np.abs(h2))
    return np.concatenate([gW1.ravel(), gW2.ravel(), gw3])


def loss_and_grads(wflat, X, target, k: int, scale: float = 1.0, round_hidden: bool = False):
    """Summed cross-entropy over cities (times `scale`), its gradient over the flat weights and
    the unscaled dz = softmax - y of every row.

    Backward pass by the chain rule: dz = softmax - y per city; dw3 = h2^T dz;
    dh2 = dz w3^T masked by [a2 > 0] (and 0 on the constant unit); dW2 = dh2^T h1;
    dh1 = dh2 W2 masked by [a1 > 0] (0 on the constant unit); dW1 = dh1^T x.  With round_hidden
    the forward pass rounds h1 and h2 to BF16 (``forward``) and the chain rule runs through the
    rounded activations, the rounding itself passed as the identity, as the kernels do."""
    W1, W2, w3 = split(wflat)
    X = np.asarray(X, np.float64)
    z, h1, h2, a1, a2 = forward(wflat, X, round_hidden)
    cities = len(target)
    zc = z.reshape(cities, k)
    y = np.zeros((cities, k))
    for c in range(cities):
        t = int(target[c])
        ranks = [r for r in range(k) if (t >> r) & 1]
        for r in ranks:
            y[c, r] = 1.0 / len(ranks)
    live = y.sum(axis=1) > 0
    mx = zc.max(axis=1, keepdims=True)
    lse = mx[:, 0] + np.log(np.exp(zc - mx).sum(axis=1))
    p = np.exp(zc - lse[:, None])
    loss = scale * float(np.sum(live * -(y * (zc - lse[:, None])).sum(axis=1)))
    dz = np.where(live[:, None], p - y, 0.0).reshape(-1)
    gw3 = h2.T @ (scale * dz)
    dh2 = np.outer(scale * dz, w3) * (a2 > 0)
    dh2[:, H - 1] = 0.0
    gW2 = dh2.T @ h1
    dh1 = (dh2 @ W2) * (a1 > 0)
    dh1[:, H - 1] = 0.0
    gW1 = dh1.T @ X
    return loss, np.concatenate([gW1.ravel(), gW2.ravel(), gw3]), dz


def adam_step(w, m1, m2, grad, mask, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015) on the masked entries; returns new (w, m1, m2)."""
    w, m1, m2, grad = (np.array(a, np.float64) for a in (w, m1, m2, grad))
    on = np.asarray(mask).astype(bool)
    m1n = np.where(on, b1 * m1 + (1 - b1) * grad, m1)
    m2n = np.where(on, b2 * m2 + (1 - b2) * grad * grad, m2)
    c1, c2 = 1 - b1 ** step, 1 - b2 ** step
    wn = np.where(on, w - lr * (m1n / c1) / (np.sqrt(m2n / c2) + eps), w)
    return wn, m1n, m2n

