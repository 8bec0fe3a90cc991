"""Seeded synthetic TSP instances: the only code shared by the oracle tests and the CUDA path.

This module draws city coordinates and nothing else. It holds none of the ACO method's
arithmetic (no distances, no pheromone, no draws the method makes): the method's own random
numbers come from a counter-based generator that the oracle and the CUDA library each
implement independently.

Instances are symmetric Euclidean TSPs on FP64 coordinates (the problem of Section 2 of
Chitty, "Applying ACO To Large Scale TSP Instances"). The paper's datasets (TSPLIB, the art
instances) are not available; these generators stand in for them with the same sizes:

* ``uniform``   -- n cities uniform in [0, 1)^2.
* ``clustered`` -- c Gaussian clusters, centres uniform in [0, 1)^2, city i in cluster i mod c,
                   standard deviation sigma, no clipping (points may leave the unit square).
* ``mixed``     -- half uniform, half clustered (the 10,000-city workload).

Every generator is a pure function of its arguments (numpy's PCG64 stream for the seed) and
returns a C-contiguous float64 array of shape (n, 2) with no two identical points.
"""
from __future__ import annotations

import numpy as np

__all__ = ["uniform", "clustered", "mixed", "make", "batch_sizes", "permutations", "snake_tours", "bf16_values",
           "mlp_weights", "edge_scores", "WORKLOADS"]


def _dedupe(xy: np.ndarray, rng: np.random.Generator, redraw) -> np.ndarray:
    """Redraw any point that repeats an earlier one (keeps the first occurrence)."""
    for _ in range(64):
        _, first = np.unique(xy, axis=0, return_index=True)
        if first.size == xy.shape[0]:
            return xy
        dup = np.setdiff1d(np.arange(xy.shape[0]), first)
        xy[dup] = redraw(dup, rng)
    raise RuntimeError("could not draw distinct points")


def uniform(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    xy = rng.random((n, 2))
    xy = _dedupe(xy, rng, lambda idx, r: r.random((idx.size, 2)))
    return np.ascontiguousarray(xy, dtype=np.float64)


def clustered(n: int, n_clusters: int, sigma: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    centres = rng.random((n_clusters, 2))
    member = np.arange(n) % n_clusters
    xy = centres[member] + sigma * rng.standard_normal((n, 2))

    def redraw(idx, r):
        return centres[member[idx]] + sigma * r.standard_normal((idx.size, 2))

    xy = _dedupe(xy, rng, redraw)
    return np.ascontiguousarray(xy, dtype=np.float64)


def mixed(n: int, n_clusters: int, sigma: float, seed: int) -> np.ndarray:
    half = n // 2
    a = uniform(half, seed)
    b = clustered(n - half, n_clusters, sigma, seed + 0x9E3779B9)
    xy = np.concatenate([a, b], axis=0)
    rng = np.random.default_rng(seed + 1)
    xy = _dedupe(xy, rng, lambda idx, r: r.random((idx.size, 2)))
    return np.ascontiguousarray(xy, dtype=np.float64)


# The workloads the library is measured and tested on (sizes from the paper's experiments and
# the stated large-scale target). ``params`` are the ACO parameters of each workload.
WORKLOADS = {
    # Section 2 plain ACO, dense pheromone matrix.
    "dense100": dict(gen=("uniform", dict(n=100, seed=1)),
                     params=dict(mode=0, n=100, m=100, k=0, alpha=1.0, beta=2.0, rho=0.5,
                                 tau0=1.0, max_mod_frac=1.0, p_partial=1.0, seed=1),
                     iterations=100),
    # Section 3 scalable variant, 10,000 cities (half uniform, half in 20 clusters).
    "lbest10k": dict(gen=("mixed", dict(n=10_000, n_clusters=20, sigma=0.02, seed=2)),
                     params=dict(mode=1, n=10_000, m=256, k=20, alpha=1.0, beta=2.0, rho=0.1,
                                 tau0=1.0, max_mod_frac=0.1, p_partial=1.0, seed=2),
                     iterations=200),
    # Section 3 scalable variant at the paper's largest size (200,000 cities, 200 clusters).
    "lbest200k": dict(gen=("clustered", dict(n=200_000, n_clusters=200, sigma=0.005, seed=3)),
                      params=dict(mode=1, n=200_000, m=1024, k=16, alpha=1.0, beta=2.0, rho=0.1,
                                  tau0=1.0, max_mod_frac=0.01, p_partial=1.0, seed=3),
                      iterations=50),
}


def make(name: str) -> np.ndarray:
    """Coordinates of a named workload."""
    kind, kw = WORKLOADS[name]["gen"]
    return {"uniform": uniform, "clustered": clustered, "mixed": mixed}[kind](**kw)


def batch_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Instance sizes log-uniform in [lo, hi] (the batched workload's ragged sizes)."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size=count))).astype(np.int64).clip(lo, hi)


# ------------------------------------------------------------------ inputs of the learned proposal
def permutations(count: int, n: int, seed: int) -> np.ndarray:
    """`count` independent uniformly random tours of n cities, int32 [count][n]."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.permutation(n) for _ in range(count)]).astype(np.int32)


def snake_tours(xy: np.ndarray, count: int, seed: int, grid: int = 512, reversals: int = 64,
                max_len: int = 2000) -> np.ndarray:
    """`count` spatially coherent random tours, int32 [count][n]: the cities in the order of a
    boustrophedon sweep over a grid x grid binning of the bounding box (by x within a bin), then
    per tour a random rotation and `reversals` reversals of random segments of 2..max_len
    positions.  (A population of tours that look like a colony's, without running one.)"""
    rng = np.random.default_rng(seed)
    n = xy.shape[0]
    lo = xy.min(axis=0)
    span = np.maximum(xy.max(axis=0) - lo, 1e-300)
    b = np.minimum(((xy - lo) / span * grid).astype(np.int64), grid - 1)
    col = np.where(b[:, 1] % 2 == 0, b[:, 0], grid - 1 - b[:, 0])
    base = np.lexsort((xy[:, 0], col, b[:, 1]))
    out = np.empty((count, n), np.int32)
    for a in range(count):
        t = np.roll(base, int(rng.integers(n)))
        for _ in range(reversals):
            i = int(rng.integers(n - 2))
            ln = int(rng.integers(2, max(3, min(max_len, n - i) + 1)))
            t[i:i + ln] = t[i:i + ln][::-1]
        out[a] = t
    return out


def bf16_values(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform values in [lo, hi) truncated to BF16 (the top 16 bits of their FP32 pattern),
    returned as float32."""
    rng = np.random.default_rng(seed)
    x = (lo + (hi - lo) * rng.random(shape)).astype(np.float32)
    return (x.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32)


def mlp_weights(seed: int, inputs: int = 16, hidden: int = 64) -> np.ndarray:
    """Initial weights of the edge-scoring network as one float32 vector (W1 [hidden][inputs],
    W2 [hidden][hidden], w3 [hidden]): zero-mean normals with He scaling (variance 2 / fan-in,
    fan-in 6 for W1 whose inputs 6.. are always zero)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, np.sqrt(2.0 / 6), (hidden, inputs))
    W2 = rng.normal(0.0, np.sqrt(2.0 / hidden), (hidden, hidden))
    w3 = rng.normal(0.0, np.sqrt(1.0 / hidden), hidden)
    return np.concatenate([W1.ravel(), W2.ravel(), w3]).astype(np.float32)


def edge_scores(n: int, k: int, seed: int) -> np.ndarray:
    """Positive float32 scores [n][k], log-uniform over six decades."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(-7.0, 7.0, (n, k))).astype(np.float32)
