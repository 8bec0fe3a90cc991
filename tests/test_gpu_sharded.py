"""One colony split by ants over several instances equals the single colony, bit for bit (GB300).

Ranks are stood in for by instances on the one GPU: each constructs its ant range, exports the
commits of its improved ants (aco_export_commits), the buffers are stacked by a device copy (what
the all-gather does between GPUs), and every instance imports all of them (aco_import_commits)
and updates.  After every iteration every instance's l_best, lengths and C_gbest equal those of
a single colony running all the ants, and the decisions summed over the instances equal its own.
"""
import numpy as np
import pytest

import aco_synth
from tests.gpu_common import require_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _stack(bufs, words):
    stride = max(words)
    stride += stride & 1
    out = torch.zeros((len(bufs), stride), dtype=torch.int32, device="cuda")
    for i, (b, w) in enumerate(zip(bufs, words)):
        out[i, :w] = b[:w]
    return out


@pytest.mark.parametrize("n,m,k,f,p_partial,ranks,iters", [
    (2000, 64, 16, 0.2, 1.0, 2, 8),   # staged rows, two ranks
    (1500, 48, 20, 0.3, 0.7, 3, 6),   # k = 20, full tours mid-run, three ranks
    (900, 37, 8, 0.5, 1.0, 4, 6),     # uneven shares
])
def test_split_colony_equals_single(n, m, k, f, p_partial, ranks, iters):
    require_gpu()
    from paper_1709_03187_gb300 import Colony, aco_export_commits, aco_import_commits, aco_set_ant_range
    from paper_1709_03187_gb300.sharded import ant_range

    xy = aco_synth.clustered(n, 10, 0.02, n + ranks)
    kw = dict(mode=1, n=n, m=m, k=k, alpha=1.0, beta=2.0, tau0=1.0, max_mod_frac=f, p_partial=p_partial, seed=n)
    single = Colony(xy, **kw)
    single.build_candidates()
    parts, bufs, caps = [], [], []
    for r in range(ranks):
        c = Colony(xy, **kw)
        c.build_candidates()
        a0, a1 = ant_range(m, r, ranks)
        aco_set_ant_range(c.handle, a0, a1)
        caps.append((a1 - a0) * (12 + n) + 4)
        bufs.append(torch.empty(caps[-1], dtype=torch.int32, device="cuda"))
        parts.append(c)
    for it in range(iters):
        single.iterate(it)
        words = []
        for c, b, cap in zip(parts, bufs, caps):
            c.construct(it)
            words.append(aco_export_commits(c.handle, b, cap))
        recs = _stack(bufs, words)
        for c in parts:
            aco_import_commits(c.handle, recs, ranks, recs.shape[1])
            c.update()
        lb, cl, _ = single.state()
        for r, c in enumerate(parts):
            lb_r, cl_r, _ = c.state()
            assert torch.equal(lb_r, lb), f"iteration {it}, rank {r}: l_best"
            assert torch.equal(cl_r, cl), f"iteration {it}, rank {r}: lengths"
    st = single.stats()
    sts = [c.stats() for c in parts]
    assert all(s["gbest"] == st["gbest"] for s in sts)
    assert sum(s["decisions"] for s in sts) == st["decisions"]
    assert sum(s["fallbacks"] for s in sts) == st["fallbacks"]
    for c in parts + [single]:
        c.close()


def test_export_capacity_and_malformed_records():
    require_gpu()
    from paper_1709_03187_gb300 import AcoError, Colony, aco_export_commits, aco_import_commits, aco_set_ant_range

    n, m = 300, 8
    xy = aco_synth.uniform(n, 4)
    c = Colony(xy, mode=1, n=n, m=m, k=8, max_mod_frac=0.3, seed=4)
    c.build_candidates()
    aco_set_ant_range(c.handle, 0, 4)
    c.construct(0)  # initial tours: four full records of n cities
    small = torch.empty(64, dtype=torch.int32, device="cuda")
    with pytest.raises(AcoError):
        aco_export_commits(c.handle, small, 64)
    buf = torch.empty(4 * (12 + n) + 4, dtype=torch.int32, device="cuda")
    words = aco_export_commits(c.handle, buf, buf.numel())
    assert words == 4 * (12 + n) + 4 and int(buf[0]) == 4
    bad = buf[:words].clone()
    bad[4] = m + 5  # an ant the colony does not have
    aco_import_commits(c.handle, bad.view(1, -1), 1, words)
    with pytest.raises(AcoError):
        c.stats()
    with pytest.raises(AcoError):
        aco_set_ant_range(c.handle, 3, 3)
    c.close()
