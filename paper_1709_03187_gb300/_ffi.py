"""ctypes declarations of include/aco.h and one Python function per entry point.

Arguments are marshalled only: tensors become device pointers, streams become cudaStream_t
handles, and a non-OK aco_status becomes ``AcoError``.  There is no fallback path: if the
shared library is missing the first call raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(HERE, "lib", "libaco_gb300.so")

ACO_MODE_DENSE = 0
ACO_MODE_LBEST_PARTIAL = 1
_STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error", 4: "call out of order",
           5: "device wait timed out"}


class AcoError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32), ("n", ctypes.c_int32), ("m", ctypes.c_int32), ("k", ctypes.c_int32),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("rho", ctypes.c_double), ("tau0", ctypes.c_double),
        ("max_mod_frac", ctypes.c_double), ("p_partial", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("fallback", ctypes.c_int32), ("selection", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("decisions", ctypes.c_uint64), ("fallbacks", ctypes.c_uint64), ("exact_resolves", ctypes.c_uint64),
        ("improved", ctypes.c_uint64), ("partial_ants", ctypes.c_uint64), ("full_ants", ctypes.c_uint64),
        ("gbest", ctypes.c_double), ("gbest_ant", ctypes.c_int32), ("iterations", ctypes.c_int32),
        ("ls_moves", ctypes.c_uint64), ("fallback_rebuilt", ctypes.c_uint64), ("fallback_scanned", ctypes.c_uint64),
        ("fallback_fast", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise ImportError(f"CUDA library not built: {library_path} (run paper_1709_03187_gb300.build.build())")
        L = ctypes.CDLL(library_path)
        V, I32, I32P = ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p
        S = ctypes.c_int
        sig = {
            "aco_create_instance": (S, [V, ctypes.POINTER(Params), V, ctypes.POINTER(V)]),
            "aco_build_candidates": (S, [V, V]),
            "aco_construct_tours": (S, [V, I32, V, V]),
            "aco_update_pheromone": (S, [V]),
            "aco_tour_lengths": (S, [V, V, I32, V]),
            "aco_get_state": (S, [V, V, V, V]),
            "aco_set_state": (S, [V, V, V]),
            "aco_get_stats": (S, [V, ctypes.POINTER(Stats)]),
            "aco_step_probs": (S, [V, I32, V, V, V]),
            "aco_destroy_instance": (None, [V]),
            "aco_build_candidates_noalloc": (S, [V, I32, I32, V, V]),
            "aco_set_ant_range": (S, [V, I32, I32]),
            "aco_export_commits": (S, [V, V, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
            "aco_import_commits": (S, [V, V, I32, ctypes.c_int64]),
            "aco_probe_bandwidth": (S, [V, ctypes.c_int64, I32, I32, V, ctypes.POINTER(ctypes.c_float)]),
            "aco_batch_create": (S, [V, V, I32, ctypes.POINTER(Params), V, ctypes.POINTER(V)]),
            "aco_batch_build_candidates": (S, [V]),
            "aco_batch_run": (S, [V, I32, I32, I32]),
            "aco_batch_get_state": (S, [V, V, V]),
            "aco_batch_get_best": (S, [V, V]),
            "aco_batch_schedule": (S, [V, V, V, V, V, V]),
            "aco_batch_set_schedule": (S, [V, I32]),
            "aco_batch_set_wait_limit": (S, [V, ctypes.c_double]),
            "aco_batch_last_error": (ctypes.c_char_p, [V]),
            "aco_batch_destroy": (None, [V]),
            "aco_batch_instance": (S, [V, I32, ctypes.POINTER(V)]),
            "aco_mlp_create": (S, [V, ctypes.c_int64, V, ctypes.POINTER(V)]),
            "aco_mlp_get_weights": (S, [V, V]),
            "aco_mlp_forward": (S, [V, V, ctypes.c_int64, V, V, ctypes.c_float]),
            "aco_mlp_backward": (S, [V, V, V, I32, I32, ctypes.c_float, V, V]),
            "aco_mlp_adam": (S, [V, V, ctypes.c_float]),
            "aco_mlp_train": (S, [V, V, V, I32, I32, I32, I32, ctypes.c_float, V]),
            "aco_mlp_last_error": (ctypes.c_char_p, [V]),
            "aco_mlp_destroy": (None, [V]),
            "aco_edge_features": (S, [V, I32, V]),
            "aco_tour_labels": (S, [V, V]),
            "aco_set_edge_scores": (S, [V, V]),
            "aco_set_max_mod_frac": (S, [V, ctypes.c_double]),
            "aco_set_p_partial": (S, [V, ctypes.c_double]),
            "aco_set_local_search": (S, [V, ctypes.c_double, I32]),
            "aco_set_async_share": (S, [V, I32]),
            "aco_status_string": (ctypes.c_char_p, [S]),
            "aco_last_error": (ctypes.c_char_p, [V]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        del I32P
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _check(status: int, where: str, handle=None):
    if status != 0:
        msg = lib().aco_last_error(handle)
        raise AcoError(status, where, msg.decode() if msg else "")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def aco_create_instance(xy_dev, params: Params, stream=None):
    h = ctypes.c_void_p()
    _check(lib().aco_create_instance(_ptr(xy_dev), ctypes.byref(params), _stream_handle(stream), ctypes.byref(h)),
           "aco_create_instance")
    return h.value


def aco_build_candidates(h, cand_out_dev=None):
    _check(lib().aco_build_candidates(h, _ptr(cand_out_dev)), "aco_build_candidates", h)


def aco_construct_tours(h, iteration: int, tours_out_dev=None, len_out_dev=None):
    _check(lib().aco_construct_tours(h, iteration, _ptr(tours_out_dev), _ptr(len_out_dev)), "aco_construct_tours", h)


def aco_update_pheromone(h):
    _check(lib().aco_update_pheromone(h), "aco_update_pheromone", h)


def aco_tour_lengths(h, tours_dev, count: int, out_dev):
    _check(lib().aco_tour_lengths(h, _ptr(tours_dev), count, _ptr(out_dev)), "aco_tour_lengths", h)


def aco_get_state(h, lbest_out_dev=None, clen_out_dev=None, tau_out_dev=None):
    _check(lib().aco_get_state(h, _ptr(lbest_out_dev), _ptr(clen_out_dev), _ptr(tau_out_dev)), "aco_get_state", h)


def aco_set_state(h, lbest_dev=None, tau_dev=None):
    _check(lib().aco_set_state(h, _ptr(lbest_dev), _ptr(tau_dev)), "aco_set_state", h)


def aco_get_stats(h) -> Stats:
    s = Stats()
    _check(lib().aco_get_stats(h, ctypes.byref(s)), "aco_get_stats", h)
    return s


def aco_step_probs(h, city: int, visited_bits_dev, probs_out_dev, exhausted_out_dev):
    _check(lib().aco_step_probs(h, city, _ptr(visited_bits_dev), _ptr(probs_out_dev), _ptr(exhausted_out_dev)),
           "aco_step_probs", h)


def _bcheck(status: int, where: str, b):
    if status != 0:
        msg = lib().aco_batch_last_error(b) if b else b""
        raise AcoError(status, where, msg.decode() if msg else "")


def aco_batch_create(xy_dev, n_host, params: Params, stream=None):
    import numpy as np

    ns = np.ascontiguousarray(n_host, dtype=np.int32)
    h = ctypes.c_void_p()
    _bcheck(lib().aco_batch_create(_ptr(xy_dev), ns.ctypes.data_as(ctypes.c_void_p), int(ns.size),
                                   ctypes.byref(params), _stream_handle(stream), ctypes.byref(h)),
            "aco_batch_create", None)
    return h.value


def aco_batch_build_candidates(b):
    _bcheck(lib().aco_batch_build_candidates(b), "aco_batch_build_candidates", b)


def aco_batch_run(b, first_iteration: int, iterations: int, tune: bool = False):
    _bcheck(lib().aco_batch_run(b, first_iteration, iterations, 1 if tune else 0), "aco_batch_run", b)


def aco_batch_get_state(b, lbest_out_dev=None, clen_out_dev=None):
    _bcheck(lib().aco_batch_get_state(b, _ptr(lbest_out_dev), _ptr(clen_out_dev)), "aco_batch_get_state", b)


def aco_batch_get_best(b, count: int):
    import numpy as np

    out = np.zeros(count, np.float64)
    _bcheck(lib().aco_batch_get_best(b, out.ctypes.data_as(ctypes.c_void_p)), "aco_batch_get_best", b)
    return out


ACO_BATCH_SCHEDULES = 12


def aco_batch_schedule(b):
    """(schedule, warps per block, min blocks per SM, ants per pull (0: four launches)), tuning ms."""
    import numpy as np

    sc, w, mb, pull = (ctypes.c_int32() for _ in range(4))
    ms = np.zeros(ACO_BATCH_SCHEDULES, np.float32)
    _bcheck(lib().aco_batch_schedule(b, ctypes.byref(sc), ctypes.byref(w), ctypes.byref(mb), ctypes.byref(pull),
                                     ms.ctypes.data_as(ctypes.c_void_p)), "aco_batch_schedule", b)
    return (int(sc.value), int(w.value), int(mb.value), int(pull.value)), ms


def aco_batch_set_schedule(b, schedule: int):
    _bcheck(lib().aco_batch_set_schedule(b, schedule), "aco_batch_set_schedule", b)


def aco_batch_set_wait_limit(b, seconds: float):
    _bcheck(lib().aco_batch_set_wait_limit(b, seconds), "aco_batch_set_wait_limit", b)


def aco_batch_destroy(b):
    if b:
        lib().aco_batch_destroy(b)


def aco_build_candidates_noalloc(xy_dev, n: int, k: int, cand_out_dev, stream=None):
    status = lib().aco_build_candidates_noalloc(_ptr(xy_dev), n, k, _ptr(cand_out_dev), _stream_handle(stream))
    if status != 0:
        raise AcoError(status, "aco_build_candidates_noalloc", "")


def aco_set_ant_range(h, ant_begin: int, ant_end: int):
    _check(lib().aco_set_ant_range(h, ant_begin, ant_end), "aco_set_ant_range", h)


def aco_export_commits(h, buf_dev, cap_words: int) -> int:
    words = ctypes.c_int64()
    _check(lib().aco_export_commits(h, _ptr(buf_dev), cap_words, ctypes.byref(words)), "aco_export_commits", h)
    return int(words.value)


def aco_import_commits(h, bufs_dev, count: int, stride_words: int):
    _check(lib().aco_import_commits(h, _ptr(bufs_dev), count, stride_words), "aco_import_commits", h)


def aco_probe_bandwidth(buf_dev, nbytes: int, mode: int, reps: int, stream=None) -> float:
    """Milliseconds for `reps` passes of the bandwidth probe over the caller's buffer (mode 0: read
    it; mode 1: copy its first half to its second half)."""
    ms = ctypes.c_float()
    status = lib().aco_probe_bandwidth(_ptr(buf_dev), nbytes, mode, reps, _stream_handle(stream), ctypes.byref(ms))
    if status != 0:
        raise AcoError(status, "aco_probe_bandwidth", "")
    return float(ms.value)


def aco_destroy_instance(h):
    if h:
        lib().aco_destroy_instance(h)


def aco_batch_instance(b, i: int):
    h = ctypes.c_void_p()
    _bcheck(lib().aco_batch_instance(b, i, ctypes.byref(h)), "aco_batch_instance", b)
    return h.value


# ------------------------------------------------------------------ learned edge proposal
ACO_MLP_WEIGHTS = 64 * 16 + 64 * 64 + 64


def _mcheck(status: int, where: str, h):
    if status != 0:
        msg = lib().aco_mlp_last_error(h) if h else b""
        raise AcoError(status, where, msg.decode() if msg else "")


def aco_mlp_create(w_host, max_rows: int, stream=None):
    import numpy as np

    w = np.ascontiguousarray(w_host, dtype=np.float32)
    if w.size != ACO_MLP_WEIGHTS:
        raise ValueError(f"expected {ACO_MLP_WEIGHTS} weights, got {w.size}")
    h = ctypes.c_void_p()
    _mcheck(lib().aco_mlp_create(w.ctypes.data_as(ctypes.c_void_p), int(max_rows), _stream_handle(stream),
                                 ctypes.byref(h)), "aco_mlp_create", None)
    return h.value


def aco_mlp_get_weights(h):
    import numpy as np

    out = np.zeros(ACO_MLP_WEIGHTS, np.float32)
    _mcheck(lib().aco_mlp_get_weights(h, out.ctypes.data_as(ctypes.c_void_p)), "aco_mlp_get_weights", h)
    return out


def aco_mlp_forward(h, X_dev, rows: int, z_dev=None, score_dev=None, beta: float = 1.0):
    _mcheck(lib().aco_mlp_forward(h, _ptr(X_dev), int(rows), _ptr(z_dev), _ptr(score_dev), beta), "aco_mlp_forward",
            h)


def aco_mlp_backward(h, X_dev, target_dev, cities: int, k: int, scale: float, grad_dev=None, loss_dev=None):
    _mcheck(lib().aco_mlp_backward(h, _ptr(X_dev), _ptr(target_dev), cities, k, scale, _ptr(grad_dev),
                                   _ptr(loss_dev)), "aco_mlp_backward", h)


def aco_mlp_adam(h, grad_dev, lr: float):
    _mcheck(lib().aco_mlp_adam(h, _ptr(grad_dev), lr), "aco_mlp_adam", h)


def aco_mlp_train(h, X_dev, target_dev, cities: int, k: int, batch_cities: int, steps: int, lr: float,
                  loss_dev=None):
    _mcheck(lib().aco_mlp_train(h, _ptr(X_dev), _ptr(target_dev), cities, k, batch_cities, steps, lr,
                                _ptr(loss_dev)), "aco_mlp_train", h)


def aco_mlp_destroy(h):
    if h:
        lib().aco_mlp_destroy(h)


def aco_edge_features(h, degree_ants: int, X_dev):
    _check(lib().aco_edge_features(h, degree_ants, _ptr(X_dev)), "aco_edge_features", h)


def aco_tour_labels(h, target_dev):
    _check(lib().aco_tour_labels(h, _ptr(target_dev)), "aco_tour_labels", h)


def aco_set_edge_scores(h, score_dev=None):
    _check(lib().aco_set_edge_scores(h, _ptr(score_dev)), "aco_set_edge_scores", h)


def aco_set_max_mod_frac(h, f: float):
    _check(lib().aco_set_max_mod_frac(h, f), "aco_set_max_mod_frac", h)


def aco_set_p_partial(h, p_partial: float):
    _check(lib().aco_set_p_partial(h, p_partial), "aco_set_p_partial", h)


def aco_set_local_search(h, p: float, window: int = 500):
    _check(lib().aco_set_local_search(h, p, window), "aco_set_local_search", h)


def aco_set_async_share(h, on: bool):
    _check(lib().aco_set_async_share(h, 1 if on else 0), "aco_set_async_share", h)
