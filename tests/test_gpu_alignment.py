"""Caller buffers that are not aligned to their element type are refused with
ACO_ERR_INVALID_ARG before anything is enqueued, and the instance keeps working afterwards
(the convention stated at the top of include/aco.h)."""
import numpy as np
import pytest

import aco_synth
from tests.gpu_common import require_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_misaligned_buffers_are_refused_and_the_instance_keeps_working():
    require_gpu()
    from paper_1709_03187_gb300 import AcoError, Colony, _ffi

    n, m, k = 300, 8, 8
    xy = aco_synth.uniform(n, 5)
    raw = torch.zeros(2 * n + 1, dtype=torch.float64, device="cuda")
    raw[1:].copy_(torch.from_numpy(xy).reshape(-1))
    as_bytes = raw.view(torch.uint8)
    odd_xy = as_bytes[4:4 + 16 * n]  # 4 bytes into an FP64 buffer
    params = _ffi.Params(mode=1, n=n, m=m, k=k, alpha=1.0, beta=2.0, rho=0.5, tau0=1.0, max_mod_frac=0.1,
                         p_partial=1.0, seed=2)
    with pytest.raises(AcoError) as e:
        _ffi.aco_create_instance(odd_xy, params)
    assert e.value.status == 1

    col = Colony(xy, mode=1, n=n, m=m, k=k, seed=2)
    col.build_candidates()
    col.iterate(0)
    tours = torch.empty((m, n), dtype=torch.int32, device="cuda")
    _ffi.aco_get_state(col.handle, tours, None, None)
    out = torch.zeros(2 * m + 1, dtype=torch.float64, device="cuda")
    odd_out = out.view(torch.uint8)[4:4 + 8 * m]
    with pytest.raises(AcoError) as e:
        _ffi.aco_tour_lengths(col.handle, tours, m, odd_out)
    assert e.value.status == 1
    with pytest.raises(AcoError) as e:
        _ffi.aco_construct_tours(col.handle, 1, None, odd_out)
    assert e.value.status == 1
    # the same call with an aligned buffer succeeds and gives the tours' lengths
    good = torch.empty(m, dtype=torch.float64, device="cuda")
    _ffi.aco_tour_lengths(col.handle, tours, m, good)
    t = tours.cpu().numpy()
    ref = np.sqrt(((xy[t] - xy[np.roll(t, -1, axis=1)]) ** 2).sum(-1)).sum(1)
    assert np.allclose(good.cpu().numpy(), ref, rtol=1e-12, atol=0)
    col.iterate(1)
    col.close()
