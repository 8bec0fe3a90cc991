"""Batch: many independent colonies of uneven size advanced together (wrapper of aco_batch_*)."""
from __future__ import annotations

import numpy as np
import torch

from . import _ffi
from .colony import make_params


class Batch:
    """Instances given as a list of (n_i, 2) coordinate arrays; shared ACO parameters.

    Instance i gets m_i = min(n_i, m) ants and seed `seed + i`.
    """

    def __init__(self, xys, *, m: int, k: int, alpha: float = 1.0, beta: float = 2.0, tau0: float = 1.0,
                 max_mod_frac: float = 1.0, p_partial: float = 1.0, seed: int = 1, fallback: int = 0,
                 selection: int = 0, stream: torch.cuda.Stream | None = None):
        self.ns = np.array([x.shape[0] for x in xys], np.int32)
        self.ms = np.minimum(self.ns, m)
        self.count = len(xys)
        self.xy = torch.from_numpy(np.ascontiguousarray(np.concatenate(xys, 0), np.float64)).cuda()
        self.params = make_params(1, int(self.ns.max()), m, k, alpha, beta, 0.0, tau0, max_mod_frac, p_partial, seed,
                                  fallback, selection)
        self.stream = stream
        self._h = _ffi.aco_batch_create(self.xy, self.ns, self.params, stream)

    def close(self):
        if self._h:
            _ffi.aco_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_candidates(self):
        _ffi.aco_batch_build_candidates(self._h)

    def run(self, first_iteration: int, iterations: int, tune: bool = False):
        _ffi.aco_batch_run(self._h, first_iteration, iterations, tune)

    def best(self) -> np.ndarray:
        return _ffi.aco_batch_get_best(self._h, self.count)

    def schedule(self):
        """((schedule, warps per block, min blocks per SM, ants per pull), tuning ms per schedule)."""
        return _ffi.aco_batch_schedule(self._h)

    def set_schedule(self, schedule: int):
        """Fix the launch schedule (0-7: four launches per iteration; 8-11: one persistent launch),
        -1 = autotune."""
        _ffi.aco_batch_set_schedule(self._h, schedule)

    def set_wait_limit(self, seconds: float):
        _ffi.aco_batch_set_wait_limit(self._h, seconds)

    def state(self):
        """Per-instance (l_best (m_i, n_i), lengths (m_i,)) as numpy arrays."""
        tot_t = int(np.sum(self.ms.astype(np.int64) * self.ns))
        lb = torch.empty(tot_t, dtype=torch.int32, device="cuda")
        cl = torch.empty(int(self.ms.sum()), dtype=torch.float64, device="cuda")
        _ffi.aco_batch_get_state(self._h, lb, cl)
        lb, cl = lb.cpu().numpy(), cl.cpu().numpy()
        out, to, ao = [], 0, 0
        for n, m in zip(self.ns, self.ms):
            out.append((lb[to:to + m * n].reshape(m, n), cl[ao:ao + m]))
            to += m * n
            ao += m
        return out
