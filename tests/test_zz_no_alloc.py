"""The allocation-free candidate-list entry point gives the regular entry point's lists.

aco_build_candidates_noalloc is for callers that cannot allocate device memory where they need
candidate lists (their device memory belongs to another allocator, or they must not allocate once
running): its working memory is a fixed array inside the library, shared by every call.  The
lists are integer results, compared bit for bit with aco_build_candidates, on two calls in a row
(the second call reuses the array after a larger first call).  This file's name sorts last so a
failure here cannot hide the other GPU tests.
"""
import numpy as np
import pytest

import aco_synth
from tests.gpu_common import require_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _regular(xy, k):
    from paper_1709_03187_gb300 import Colony

    col = Colony(xy, mode=1, n=xy.shape[0], m=1, k=k)
    cand = col.build_candidates(return_lists=True)
    col.close()
    return cand


def test_noalloc_matches_regular_on_two_calls_in_a_row():
    require_gpu()
    from paper_1709_03187_gb300 import aco_build_candidates_noalloc

    # the largest size the array holds first, then a smaller one that reuses what it left behind
    cases = [(aco_synth.uniform(65_536, 8), 8), (aco_synth.clustered(20_000, 40, 0.01, 5), 16),
             (aco_synth.uniform(3_001, 6), 20)]
    for xy, k in cases:
        n = xy.shape[0]
        dev = torch.from_numpy(xy).cuda()
        out = torch.full((n, k), -1, dtype=torch.int32, device="cuda")
        aco_build_candidates_noalloc(dev, n, k, out)
        ref = _regular(xy, k)
        assert torch.equal(out, ref), f"n={n}: lists differ from aco_build_candidates"


def test_noalloc_rejects_what_its_array_cannot_hold():
    require_gpu()
    from paper_1709_03187_gb300 import AcoError, aco_build_candidates_noalloc

    big = torch.zeros((65_537, 2), dtype=torch.float64, device="cuda")
    out = torch.empty((65_537, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(AcoError) as e:
        aco_build_candidates_noalloc(big, 65_537, 4, out)
    assert e.value.status == 1
    xy = aco_synth.uniform(100, 1)
    xy[7] = xy[3]  # coincident cities
    dev = torch.from_numpy(xy).cuda()
    out = torch.empty((100, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(AcoError):
        aco_build_candidates_noalloc(dev, 100, 8, out)
    with pytest.raises(AcoError):
        aco_build_candidates_noalloc(dev, 100, 33, torch.empty((100, 33), dtype=torch.int32, device="cuda"))
    # non-finite coordinates are reported (the grid is then a unit box and every index clamped)
    for bad in (float("nan"), float("inf")):
        xy = aco_synth.uniform(100, 2)
        xy[11, 1] = bad
        with pytest.raises(AcoError) as e:
            aco_build_candidates_noalloc(torch.from_numpy(xy).cuda(), 100, 8, out)
        assert e.value.status == 1
    # and a valid call right after the rejected ones gives the regular lists again
    xy = aco_synth.uniform(500, 3)
    good = torch.empty((500, 8), dtype=torch.int32, device="cuda")
    aco_build_candidates_noalloc(torch.from_numpy(xy).cuda(), 500, 8, good)
    assert torch.equal(good, _regular(xy, 8))


def test_noalloc_refuses_a_capturing_stream():
    """The call synchronises and reads its error flag back, so it cannot be captured in a CUDA
    graph: on a capturing stream it returns ACO_ERR_INVALID_ARG, enqueues nothing and leaves the
    capture intact; afterwards the stream takes it normally."""
    require_gpu()
    from paper_1709_03187_gb300 import AcoError, aco_build_candidates_noalloc

    xy = aco_synth.uniform(500, 4)
    dev = torch.from_numpy(xy).cuda()
    out = torch.full((500, 8), -7, dtype=torch.int32, device="cuda")
    side = torch.zeros(4, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.graph(g, stream=s):
        side.add_(1.0)
        try:
            aco_build_candidates_noalloc(dev, 500, 8, out, stream=s)
        except AcoError as e:
            status = e.status
    assert status == 1
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(side, torch.ones(4, device="cuda"))
    assert bool((out == -7).all())  # nothing ran
    aco_build_candidates_noalloc(dev, 500, 8, out, stream=s)
    s.synchronize()
    assert torch.equal(out, _regular(xy, 8))
