"""CPU oracle for the ACO hot path (test infrastructure only).

The oracle is the correctness reference the CUDA library is checked against: a plain,
single-threaded FP64 C implementation (``aco_oracle.c``) of Chitty's ACO method -- Section 2
(Eq. 1-5, dense pheromone), Section 3 (per-ant l_best pheromone source, weights
C_gbest / C_lbest) and Algorithm 1 (PartialACO) -- plus exact k-nearest-neighbour candidate
lists and exact tour lengths.  Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package; the library never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aco_oracle.c")
_LIB_DIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_DENSE = 0
MODE_LBEST = 1


class Params(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32), ("n", ctypes.c_int32), ("m", ctypes.c_int32), ("k", ctypes.c_int32),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("rho", ctypes.c_double),
        ("tau0", ctypes.c_double), ("max_mod_frac", ctypes.c_double), ("p_partial", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("fallback", ctypes.c_int32), ("selection", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, FP64, no FMA contraction) into oracle/lib/liboracle.so."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_LIB_DIR, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        sig = {
            "or_philox4x32_10": (None, [u32p, u32p, u32p]),
            "or_u53": (ctypes.c_double, [ctypes.c_uint32, ctypes.c_uint32]),
            "or_bounded": (ctypes.c_uint32, [ctypes.c_uint32, ctypes.c_uint32]),
            "or_powr": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
            "or_edge_len": (ctypes.c_double, [f64p, ctypes.c_int, ctypes.c_int]),
            "or_tour_length": (ctypes.c_double, [ctypes.c_int, f64p, i32p]),
            "or_tour_lengths": (None, [ctypes.c_int, f64p, i32p, ctypes.c_int, f64p]),
            "or_knn": (ctypes.c_int, [ctypes.c_int, f64p, ctypes.c_int, i32p]),
            "or_create": (P, [ctypes.POINTER(Params), f64p]),
            "or_destroy": (None, [P]),
            "or_construct": (None, [P, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
            "or_construct_ex": (None, [P, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
            "or_construct_mt": (None, [P, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "or_update": (None, [P]),
            "or_get_lbest": (None, [P, i32p]),
            "or_get_clen": (None, [P, f64p]),
            "or_get_newtours": (None, [P, i32p]),
            "or_get_newlen": (None, [P, f64p]),
            "or_get_seg": (None, [P, i32p, i32p]),
            "or_get_tau": (None, [P, f64p]),
            "or_set_tau": (None, [P, f64p]),
            "or_get_cand": (None, [P, i32p]),
            "or_get_etab": (None, [P, f64p]),
            "or_get_counters": (None, [P, i64p]),
            "or_reset_counters": (None, [P]),
            "or_initialized": (ctypes.c_int, [P]),
            "or_cand_weights": (None, [P, f64p, u64p, u64p]),
            "or_set_lbest": (None, [P, i32p, f64p]),
            "or_step_probs": (ctypes.c_int, [P, ctypes.c_int, u8p, f64p]),
            "or_knn_one": (None, [ctypes.c_int, f64p, ctypes.c_int, ctypes.c_int, i32p]),
            "or_knn_sweep": (ctypes.c_int, [ctypes.c_int, f64p, ctypes.c_int, i32p]),
            "or_create_with_cand": (P, [ctypes.POINTER(Params), f64p, i32p]),
            "or_set_edge_scores": (None, [P, ctypes.c_void_p]),
            "or_set_max_mod_frac": (None, [P, ctypes.c_double]),
            "or_set_local_search": (None, [P, ctypes.c_double, ctypes.c_int]),
            "or_ls_moves": (ctypes.c_int64, [P]),
            "or_two_opt_windowed": (ctypes.c_int, [ctypes.c_int, f64p, i32p, ctypes.c_int, ctypes.c_int]),
            "or_set_p_partial": (None, [P, ctypes.c_double]),
            "or_set_newtour": (None, [P, ctypes.c_int, i32p, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
            "or_clear_built": (None, [P]),
            "or_exhausted_step": (ctypes.c_int, [P, ctypes.c_int, u8p, ctypes.c_double, ctypes.c_void_p]),
            "or_ir_pick": (ctypes.c_int, [f64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_uint32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ------------------------------------------------------------------ free functions
def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def u53(x0: int, x1: int) -> float:
    return lib().or_u53(x0, x1)


def bounded(x: int, r: int) -> int:
    return lib().or_bounded(x, r)


def ir_pick(w, seed: int, t: int, ant: int, iteration: int) -> int:
    """Independent Roulette over one candidate row of weights (rank order): the rank picked, or -1."""
    w = np.ascontiguousarray(w, np.float64)
    return int(lib().or_ir_pick(w, w.size, seed, t, ant, iteration))


def two_opt_windowed(xy: np.ndarray, tour: np.ndarray, window: int, max_passes: int = 16):
    """Windowed 2-opt of one tour (returns (improved tour, moves))."""
    t = np.ascontiguousarray(tour, np.int32).copy()
    mv = lib().or_two_opt_windowed(t.size, np.ascontiguousarray(xy, np.float64), t, window, max_passes)
    return t, int(mv)


def powr(x: float, e: float) -> float:
    return lib().or_powr(x, e)


def edge_len(xy: np.ndarray, i: int, j: int) -> float:
    return lib().or_edge_len(np.ascontiguousarray(xy, np.float64), i, j)


def tour_length(xy: np.ndarray, tour: np.ndarray) -> float:
    xy = np.ascontiguousarray(xy, np.float64)
    return lib().or_tour_length(xy.shape[0], xy, np.ascontiguousarray(tour, np.int32))


def tour_lengths(xy: np.ndarray, tours: np.ndarray) -> np.ndarray:
    xy = np.ascontiguousarray(xy, np.float64)
    tours = np.ascontiguousarray(tours, np.int32)
    out = np.zeros(tours.shape[0], np.float64)
    lib().or_tour_lengths(tours.shape[1], xy, tours, tours.shape[0], out)
    return out


def knn(xy: np.ndarray, k: int) -> np.ndarray:
    """Exact candidate lists (n, k); raises on coincident cities."""
    xy = np.ascontiguousarray(xy, np.float64)
    cand = np.zeros((xy.shape[0], k), np.int32)
    if lib().or_knn(xy.shape[0], xy, k, cand) != 0:
        raise ValueError("coincident cities")
    return cand


def knn_one(xy: np.ndarray, k: int, i: int) -> np.ndarray:
    """Candidate list of city i by brute force (sampled checks at large n)."""
    xy = np.ascontiguousarray(xy, np.float64)
    row = np.zeros(k, np.int32)
    lib().or_knn_one(xy.shape[0], xy, k, i, row)
    return row


def knn_sweep(xy: np.ndarray, k: int) -> np.ndarray:
    """Exact candidate lists by an x-sweep (same keys and result as ``knn``; fast at large n)."""
    xy = np.ascontiguousarray(xy, np.float64)
    cand = np.zeros((xy.shape[0], k), np.int32)
    if lib().or_knn_sweep(xy.shape[0], xy, k, cand) != 0:
        raise ValueError("coincident cities")
    return cand


# ------------------------------------------------------------------ solver
class Oracle:
    """One colony: dense Section 2 ACO (mode 0) or the Section 3 l_best/PartialACO form (mode 1).

    ``cand`` (mode 1 only) supplies precomputed candidate lists (from ``knn`` or ``knn_sweep``)
    instead of the O(n^2) brute force inside the oracle.
    """

    def __init__(self, xy: np.ndarray, *, mode: int, n: int, m: int, k: int = 0, alpha: float = 1.0,
                 beta: float = 2.0, rho: float = 0.5, tau0: float = 1.0, max_mod_frac: float = 1.0,
                 p_partial: float = 1.0, seed: int = 1, fallback: int = 0, selection: int = 0, cand=None):
        self.xy = np.ascontiguousarray(xy, np.float64)
        assert self.xy.shape == (n, 2)
        self.p = Params(mode, n, m, k, alpha, beta, rho, tau0, max_mod_frac, p_partial, seed, fallback, selection)
        self.n, self.m, self.k, self.mode = n, m, k, mode
        if cand is not None:
            self._h = lib().or_create_with_cand(ctypes.byref(self.p), self.xy, np.ascontiguousarray(cand, np.int32))
        else:
            self._h = lib().or_create(ctypes.byref(self.p), self.xy)
        if not self._h:
            raise ValueError("oracle rejected the instance (n < 3, bad k or coincident cities)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def construct(self, iteration: int, ants=None, rebuild: bool = True, threads: int = 1):
        """Build new tours (all ants, or the listed ones).  rebuild=False reuses the pheromone of
        the previous call (valid while the l_best population is unchanged).  threads > 1 spreads
        the ants over host threads (same result)."""
        if ants is None:
            lib().or_construct_mt(self._h, iteration, None, 0, int(rebuild), threads)
        else:
            a = np.ascontiguousarray(ants, np.int32)
            lib().or_construct_mt(self._h, iteration, a.ctypes.data_as(ctypes.c_void_p), a.size, int(rebuild),
                                  threads)

    def update(self):
        lib().or_update(self._h)

    def iterate(self, iteration: int):
        self.construct(iteration)
        self.update()

    @property
    def lbest(self) -> np.ndarray:
        out = np.zeros((self.m, self.n), np.int32)
        lib().or_get_lbest(self._h, out)
        return out

    @property
    def clen(self) -> np.ndarray:
        out = np.zeros(self.m, np.float64)
        lib().or_get_clen(self._h, out)
        return out

    @property
    def newtours(self) -> np.ndarray:
        out = np.zeros((self.m, self.n), np.int32)
        lib().or_get_newtours(self._h, out)
        return out

    @property
    def newlen(self) -> np.ndarray:
        out = np.zeros(self.m, np.float64)
        lib().or_get_newlen(self._h, out)
        return out

    def segments(self):
        s = np.zeros(self.m, np.int32)
        M = np.zeros(self.m, np.int32)
        lib().or_get_seg(self._h, s, M)
        return s, M

    @property
    def tau(self) -> np.ndarray:
        out = np.zeros((self.n, self.n), np.float64)
        lib().or_get_tau(self._h, out)
        return out

    def set_tau(self, tau: np.ndarray):
        lib().or_set_tau(self._h, np.ascontiguousarray(tau, np.float64))

    @property
    def cand(self) -> np.ndarray:
        out = np.zeros((self.n, self.k), np.int32)
        lib().or_get_cand(self._h, out)
        return out

    @property
    def etab(self) -> np.ndarray:
        out = np.zeros((self.n, self.n) if self.mode == 0 else (self.n, self.k), np.float64)
        lib().or_get_etab(self._h, out)
        return out

    def counters(self) -> dict:
        """decisions, exhausted-list steps (fallbacks), weights evaluated (scans), and exhausted-list
        picks whose pheromone lies above tau0 (boosted: an l_best neighbour outside the list)."""
        out = np.zeros(4, np.int64)
        lib().or_get_counters(self._h, out)
        return dict(decisions=int(out[0]), fallbacks=int(out[1]), scans=int(out[2]), boosted=int(out[3]))

    def reset_counters(self):
        lib().or_reset_counters(self._h)

    @property
    def initialized(self) -> bool:
        return bool(lib().or_initialized(self._h))

    def cand_weights(self):
        """(W, Q, q): candidate-edge weights tau^alpha eta^beta, integer pheromone sums, per-ant q."""
        W = np.zeros((self.n, self.k), np.float64)
        Q = np.zeros((self.n, self.k), np.uint64)
        q = np.zeros(self.m, np.uint64)
        lib().or_cand_weights(self._h, W, Q, q)
        return W, Q, q

    def set_lbest(self, lbest: np.ndarray, clen: np.ndarray):
        lib().or_set_lbest(self._h, np.ascontiguousarray(lbest, np.int32), np.ascontiguousarray(clen, np.float64))

    def set_local_search(self, p: float, window: int = 500):
        lib().or_set_local_search(self._h, p, window)

    @property
    def ls_moves(self) -> int:
        return int(lib().or_ls_moves(self._h))

    def set_max_mod_frac(self, f: float):
        lib().or_set_max_mod_frac(self._h, f)

    def set_p_partial(self, p: float):
        lib().or_set_p_partial(self._h, p)

    def set_edge_scores(self, score):
        """Learned proposal: score[i, r] replaces eta^beta on candidate edge (i, cand[i, r]); None
        restores the plain heuristic."""
        if score is None:
            lib().or_set_edge_scores(self._h, None)
            return
        s = np.ascontiguousarray(score, np.float64).reshape(self.n, self.k)
        if not np.all(np.isfinite(s)) or not np.all(s > 0):
            raise ValueError("edge scores must be finite and > 0")
        lib().or_set_edge_scores(self._h, s.ctypes.data)

    # ---- a colony split over processes by ants (the records of the library's commit exchange:
    # ant, s, P, M, start, L, new length as two words, four words of exact length (zero here:
    # the oracle measures lengths itself), then L cities; buffer header of four words)
    def export_commits(self, a0: int, a1: int) -> np.ndarray:
        """Records of ants a0..a1-1 built by the last construct whose new tour is strictly shorter
        than their l_best."""
        tours, lens, clen = self.newtours, self.newlen, self.clen
        s_arr, M_arr = self.segments()
        words = [0, 0, 0, 0]
        recs = 0
        for a in range(a0, a1):
            if not lens[a] < clen[a]:
                continue
            s, M, n = int(s_arr[a]), int(M_arr[a]), self.n
            seg = tours[a][(s + (n - M) + np.arange(M)) % n] if s >= 0 else tours[a]
            start = int(tours[a][s]) if s >= 0 else int(tours[a][0])
            bits = np.array([lens[a]], np.float64).view(np.int32)
            words += [a, s, n - M if s >= 0 else 0, M, start, len(seg), int(bits[0]), int(bits[1]), 0, 0, 0, 0]
            words += [int(c) for c in seg]
            recs += 1
        out = np.array(words, np.int64).astype(np.int32)
        out[0] = recs
        out[2:4] = np.array([out.size], np.int64).view(np.int32)
        return out

    def import_commits(self, bufs, a0: int, a1: int):
        """Sets the new tours of every record outside a0..a1 (the own ants keep theirs); ants that
        are neither own nor recorded commit nothing."""
        own = self.newtours[a0:a1].copy()
        own_len, (own_s, own_M) = self.newlen[a0:a1].copy(), self.segments()
        lib().or_clear_built(self._h)
        lb = self.lbest
        for a in range(a0, a1):
            lib().or_set_newtour(self._h, a, np.ascontiguousarray(own[a - a0]), float(own_len[a - a0]),
                                 int(own_s[a]), int(own_M[a]))
        for b in bufs:
            b = np.asarray(b, np.int32)
            recs, pos = int(b[0]), 4
            for _ in range(recs):
                a, s, P, M, start, L = (int(x) for x in b[pos:pos + 6])
                ln = float(b[pos + 6:pos + 8].copy().view(np.float64)[0])
                seg = b[pos + 12:pos + 12 + L]
                pos += 12 + L
                if a0 <= a < a1:
                    continue
                if s >= 0:
                    t = lb[a].copy()
                    t[(s + P + np.arange(M)) % self.n] = seg
                else:
                    t = seg.copy()
                lib().or_set_newtour(self._h, a, np.ascontiguousarray(t, np.int32), ln, s, M)

    def exhausted_step(self, i: int, visited: np.ndarray, u: float = 0.0):
        """The exhausted-list rule at city i (mode 1) for the given visited set and draw u, as a
        construction applies it: (city picked, weight of every city with 0 for visited ones)."""
        v = np.ascontiguousarray(visited, np.uint8)
        w = np.zeros(self.n, np.float64)
        j = lib().or_exhausted_step(self._h, i, v, float(u), w.ctypes.data)
        return int(j), w

    def step_probs(self, i: int, visited: np.ndarray):
        """Eq. 1 probabilities at city i; returns (probs, exhausted)."""
        v = np.ascontiguousarray(visited, np.uint8)
        out = np.zeros(self.n if self.mode == 0 else self.k, np.float64)
        ex = lib().or_step_probs(self._h, i, v, out)
        return out, bool(ex)
