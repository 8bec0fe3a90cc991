"""Helpers shared by the GPU tests: library build, colony pairs (CUDA path, oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

_built = False


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    global _built
    if not _built:
        from paper_1709_03187_gb300 import build

        build.build()
        _built = True


def pair(xy, **kw):
    """(CUDA colony, oracle) on the same coordinates and parameters."""
    import oracle
    from paper_1709_03187_gb300 import Colony

    require_gpu()
    col = Colony(xy, **kw)
    okw = dict(kw)
    ref = oracle.Oracle(xy, **okw)
    return col, ref


def first_divergence(a: np.ndarray, b: np.ndarray):
    idx = np.argwhere(a != b)
    return None if idx.size == 0 else tuple(idx[0])


def exact_tour_lengths(xy: np.ndarray, tours: np.ndarray) -> np.ndarray:
    """Lengths of closed tours, written here independently of the oracle, for checking tours that
    the device built: each edge's FP64 length sqrt(dx*dx + dy*dy) is placed exactly on the
    2^-96 grid (round half to even), the edges are summed as integers and the sum is rounded
    once to FP64."""
    from fractions import Fraction

    out = np.empty(len(tours))
    for a, t in enumerate(np.asarray(tours)):
        p, q = xy[t], xy[np.roll(t, -1)]
        dx, dy = p[:, 0] - q[:, 0], p[:, 1] - q[:, 1]
        d = np.sqrt(dx * dx + dy * dy)
        mant, ex = np.frexp(d)  # d = mant 2^ex, 0.5 <= mant < 1 (or d = 0)
        mi = (mant * 2.0 ** 53).astype(np.int64)  # exact: d 2^96 = mi 2^(ex + 43)
        sh = ex.astype(np.int64) + 43
        total = 0
        for s in np.unique(sh):
            sel = mi[sh == s]
            if s >= 0:  # an integer on the grid: sums of at most 512 values fit in int64
                part = sum(int(v) for v in np.add.reduceat(sel, np.arange(0, sel.size, 512)))
                total += part << int(s)
            else:  # below the grid's resolution: round each edge half to even
                total += sum(round(Fraction(int(v), 1 << int(-s))) for v in sel)
        out[a] = total / 2 ** 96  # one correctly rounded division
    return out
