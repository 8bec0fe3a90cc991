"""Colony: a convenience wrapper around one aco_instance (device tensors in, device tensors out)."""
from __future__ import annotations

import torch

from . import _ffi
from ._ffi import ACO_MODE_DENSE, ACO_MODE_LBEST_PARTIAL, Params


def make_params(mode: int, n: int, m: int, k: int = 0, alpha: float = 1.0, beta: float = 2.0, rho: float = 0.1,
                tau0: float = 1.0, max_mod_frac: float = 1.0, p_partial: float = 1.0, seed: int = 1,
                fallback: int = 0, selection: int = 0) -> Params:
    return Params(mode, n, m, k, alpha, beta, rho, tau0, max_mod_frac, p_partial, seed, fallback, selection)


def linear_f_schedule(f0: float, f1: float, ramp: int):
    """The growing modification limit of Section 7's proposal: f(t) = f0 + (f1 - f0) min(1, t / ramp)."""
    def f(t: int) -> float:
        return f0 + (f1 - f0) * min(1.0, t / ramp) if ramp > 0 else f1
    return f


class Colony:
    """One ACO colony on the current CUDA device.

    ``xy``: (n, 2) float64 coordinates (host or device); parameters as in ``aco_params``.
    """

    def __init__(self, xy, *, mode: int, n: int, m: int, k: int = 0, alpha: float = 1.0, beta: float = 2.0,
                 rho: float = 0.1, tau0: float = 1.0, max_mod_frac: float = 1.0, p_partial: float = 1.0,
                 seed: int = 1, fallback: int = 0, selection: int = 0, stream: torch.cuda.Stream | None = None,
                 device=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.xy = torch.as_tensor(xy, dtype=torch.float64).to(self.device).contiguous()
        assert self.xy.shape == (n, 2)
        self.params = make_params(mode, n, m, k, alpha, beta, rho, tau0, max_mod_frac, p_partial, seed, fallback,
                                  selection)
        self.n, self.m, self.k, self.mode = n, m, k, mode
        self.stream = stream
        self._h = None
        with torch.cuda.device(self.device):
            self._h = _ffi.aco_create_instance(self.xy, self.params, stream)

    def close(self):
        if self._h:
            _ffi.aco_destroy_instance(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def build_candidates(self, return_lists: bool = False):
        out = torch.empty((self.n, self.k), dtype=torch.int32, device=self.device) if return_lists else None
        _ffi.aco_build_candidates(self._h, out)
        return out

    def construct(self, iteration: int, return_tours: bool = False, return_lengths: bool = False):
        tours = torch.empty((self.m, self.n), dtype=torch.int32, device=self.device) if return_tours else None
        lens = torch.empty(self.m, dtype=torch.float64, device=self.device) if return_lengths else None
        _ffi.aco_construct_tours(self._h, iteration, tours, lens)
        return tours, lens

    def update(self):
        _ffi.aco_update_pheromone(self._h)

    def set_max_mod_frac(self, f: float):
        _ffi.aco_set_max_mod_frac(self._h, f)

    def set_local_search(self, p: float, window: int = 500):
        _ffi.aco_set_local_search(self._h, p, window)

    def set_p_partial(self, p_partial: float):
        _ffi.aco_set_p_partial(self._h, p_partial)

    def set_async_share(self, on: bool):
        """Asynchronous l_best sharing (improved partial rebuilds commit inside the construction
        launch; not reproducible run to run)."""
        _ffi.aco_set_async_share(self._h, on)

    def iterate(self, iteration: int):
        _ffi.aco_construct_tours(self._h, iteration, None, None)
        _ffi.aco_update_pheromone(self._h)

    def tour_lengths(self, tours: torch.Tensor) -> torch.Tensor:
        tours = tours.to(device=self.device, dtype=torch.int32).contiguous()
        out = torch.empty(tours.shape[0], dtype=torch.float64, device=self.device)
        _ffi.aco_tour_lengths(self._h, tours, tours.shape[0], out)
        return out

    def state(self):
        """(l_best or last tours (m, n), lengths (m,), tau (n, n) in dense mode else None)."""
        lb = torch.empty((self.m, self.n), dtype=torch.int32, device=self.device)
        cl = torch.empty(self.m, dtype=torch.float64, device=self.device)
        tau = torch.empty((self.n, self.n), dtype=torch.float64, device=self.device) if self.mode == ACO_MODE_DENSE else None
        _ffi.aco_get_state(self._h, lb, cl, tau)
        return lb, cl, tau

    def set_state(self, lbest=None, tau=None):
        if lbest is not None:
            lbest = torch.as_tensor(lbest, dtype=torch.int32).to(self.device).contiguous()
        if tau is not None:
            tau = torch.as_tensor(tau, dtype=torch.float64).to(self.device).contiguous()
        _ffi.aco_set_state(self._h, lbest, tau)

    def stats(self) -> dict:
        return _ffi.aco_get_stats(self._h).as_dict()

    def step_probs(self, city: int, visited_mask) -> tuple:
        """Eq. 1 probabilities as the kernel sees them; visited_mask: bool/uint8 array of n."""
        import numpy as np

        v = np.asarray(visited_mask, dtype=bool)
        words = np.zeros((self.n + 31) // 32, dtype=np.uint32)
        idx = np.nonzero(v)[0]
        np.bitwise_or.at(words, idx >> 5, (np.uint32(1) << (idx & 31).astype(np.uint32)))
        bits = torch.from_numpy(words.view(np.int32)).to(self.device)
        size = self.k if self.mode == ACO_MODE_LBEST_PARTIAL else self.n
        probs = torch.empty(size, dtype=torch.float32, device=self.device)
        ex = torch.empty(1, dtype=torch.int32, device=self.device)
        _ffi.aco_step_probs(self._h, city, bits, probs, ex)
        return probs, bool(ex.item())
