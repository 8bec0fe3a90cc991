"""EdgeScorer: the learned edge proposal (wrapper of aco_mlp_* and the instance-side calls).

A 3-layer network over per-candidate-edge features scores every candidate edge; exp(z) is the
learned counterpart of eta, and exp(z)^beta replaces eta^beta of Eq. 1 on candidate edges, while
the plain heuristic stays in place everywhere else.
Training uses the best tours that the plain method itself finds: the labels of a city are the
candidate ranks of its two neighbours in the best l_best tour.  Features, forward pass, loss,
backward pass and the optimiser all run in the library's kernels; this module only moves
pointers and loops over instances.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _ffi
from .batch import Batch

FEATURES = 16


class EdgeScorer:
    """The network and its optimiser state on the current CUDA device.

    ``weights``: ACO_MLP_WEIGHTS float32 initial weights (W1 [64][16], W2 [64][64], w3 [64]).
    ``max_rows``: the most candidate-edge rows of one backward pass or training batch."""

    def __init__(self, weights, max_rows: int = 1 << 16, stream: torch.cuda.Stream | None = None):
        self.max_rows = int(max_rows)
        self.stream = stream
        self._h = _ffi.aco_mlp_create(np.asarray(weights, np.float32), self.max_rows, stream)

    def close(self):
        if self._h:
            _ffi.aco_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def weights(self) -> np.ndarray:
        return _ffi.aco_mlp_get_weights(self._h)

    # -------------------------------------------------------------- network calls
    def forward(self, X: torch.Tensor, z: bool = True, score: bool = False, beta: float = 1.0):
        """z and/or score = exp(beta z) per row."""
        rows = X.shape[0]
        zt = torch.empty(rows, dtype=torch.float32, device=X.device) if z else None
        st = torch.empty(rows, dtype=torch.float32, device=X.device) if score else None
        _ffi.aco_mlp_forward(self._h, X, rows, zt, st, beta)
        return zt if not score else (st if not z else (zt, st))

    def backward(self, X: torch.Tensor, target: torch.Tensor, k: int, scale: float = 1.0):
        """(gradient of scale * summed loss, scaled loss) as device tensors."""
        cities = target.shape[0]
        g = torch.empty(_ffi.ACO_MLP_WEIGHTS, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _ffi.aco_mlp_backward(self._h, X, target, cities, k, scale, g, loss)
        return g, loss

    def adam(self, grad: torch.Tensor | None, lr: float):
        _ffi.aco_mlp_adam(self._h, grad, lr)

    def train(self, X: torch.Tensor, target: torch.Tensor, k: int, *, batch_cities: int, steps: int,
              lr: float) -> torch.Tensor:
        """`steps` Adam steps over the data in order; returns the per-step mean loss (device)."""
        loss = torch.empty(max(steps, 1), dtype=torch.float32, device=X.device)
        _ffi.aco_mlp_train(self._h, X, target, target.shape[0], k, batch_cities, steps, lr, loss)
        return loss[:steps]

    # -------------------------------------------------------------- instance side
    @staticmethod
    def features(handle, n: int, k: int, degree_ants: int = 16, out: torch.Tensor | None = None) -> torch.Tensor:
        X = out if out is not None else torch.empty((n * k, FEATURES), dtype=torch.bfloat16, device="cuda")
        _ffi.aco_edge_features(handle, degree_ants, X)
        return X

    @staticmethod
    def labels(handle, n: int, out: torch.Tensor | None = None) -> torch.Tensor:
        T = out if out is not None else torch.empty(n, dtype=torch.int32, device="cuda")
        _ffi.aco_tour_labels(handle, T)
        return T

    def score(self, handle, n: int, k: int, degree_ants: int = 16, beta: float = 2.0) -> torch.Tensor:
        """Features of the instance's candidate edges and the network's scores exp(z)^beta (beta:
        the instance's Eq. 1 exponent of eta), installed in place of eta^beta.  Returns the scores
        (n * k float32)."""
        X = self.features(handle, n, k, degree_ants)
        s = self.forward(X, z=False, score=True, beta=beta)
        _ffi.aco_set_edge_scores(handle, s)
        return s

    @staticmethod
    def plain(handle):
        """Restore eta^beta on the instance's candidate edges."""
        _ffi.aco_set_edge_scores(handle, None)


def training_data(xys, *, m: int, k: int, iterations: int, degree_ants: int = 16, max_mod_frac: float = 1.0,
                  seed: int = 1, tune: bool = True):
    """Run the plain method on every instance (one batch) and return (X, target):

    X: the features of every candidate edge, taken after the initial tours (the degree count then
    covers the same kind of tours that the scorer sees at inference); target: per city the
    candidate ranks of its neighbours in the best tour after `iterations` iterations."""
    b = Batch(xys, m=m, k=k, max_mod_frac=max_mod_frac, seed=seed)
    try:
        b.build_candidates()
        b.run(0, 1)
        ns = b.ns.astype(np.int64)
        X = torch.empty((int(ns.sum()) * k, FEATURES), dtype=torch.bfloat16, device="cuda")
        T = torch.empty(int(ns.sum()), dtype=torch.int32, device="cuda")
        handles = [_ffi.aco_batch_instance(b._h, i) for i in range(b.count)]
        torch.cuda.synchronize()
        off = 0
        for h, n in zip(handles, ns):
            _ffi.aco_edge_features(h, min(degree_ants, int(min(n, m))), X[off * k:(off + n) * k])
            off += n
        if iterations > 1:
            b.run(1, iterations - 1, tune=tune)
        off = 0
        for h, n in zip(handles, ns):
            _ffi.aco_tour_labels(h, T[off:off + n])
            off += n
        best = b.best()  # synchronises the batch's stream
        torch.cuda.synchronize()
        return X, T, best
    finally:
        b.close()
