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
