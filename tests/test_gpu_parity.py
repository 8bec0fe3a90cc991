"""CUDA path vs oracle, element by element, through the C ABI (needs a GB300).

Bars: candidate lists, tours and l_best bit-exact; tour lengths bit-exact (exact-sum definition,
well inside the 1e-9 relative bar); Eq. 1 probabilities within 1e-5 absolute of the oracle's FP64
values; decisions identical (the FP32 screen defers to an exact FP64 wheel near boundaries, so
the mismatch count must be zero).
"""
import math

import numpy as np
import pytest

import aco_synth
import oracle
from tests.gpu_common import first_divergence, pair, require_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LB = 1  # ACO_MODE_LBEST_PARTIAL
DENSE = 0


def _lbest_kw(n, m, k, f=0.3, seed=3, p_partial=1.0, fallback=0, alpha=1.0, beta=2.0):
    return dict(mode=LB, n=n, m=m, k=k, alpha=alpha, beta=beta, tau0=1.0, max_mod_frac=f, p_partial=p_partial,
                seed=seed, fallback=fallback)


# ------------------------------------------------------------------ candidate lists
@pytest.mark.parametrize("gen,n,k", [("uniform", 3000, 16), ("clustered", 5000, 20), ("mixed", 4000, 12),
                                     ("lattice", 400, 8), ("uniform", 5, 4), ("uniform", 33, 32),
                                     # above 8,192 cities the lists are the prefix of the 128-nearest lists
                                     ("clustered", 9000, 32), ("lattice", 10000, 16)])
def test_candidate_lists_bit_exact(gen, n, k):
    if gen == "uniform":
        xy = aco_synth.uniform(n, 11)
    elif gen == "clustered":
        xy = aco_synth.clustered(n, 17, 0.01, 12)
    elif gen == "mixed":
        xy = aco_synth.mixed(n, 20, 0.02, 13)
    else:
        g = np.arange(int(round(n ** 0.5)), dtype=np.float64)
        xy = np.ascontiguousarray(np.stack(np.meshgrid(g, g), -1).reshape(-1, 2))
    col, ref = pair(xy, **_lbest_kw(n, 2, k))
    cand = col.build_candidates(return_lists=True).cpu().numpy()
    assert first_divergence(cand, ref.cand) is None


def test_duplicate_cities_rejected():
    from paper_1709_03187_gb300 import AcoError

    xy = aco_synth.uniform(50, 1)
    xy[17] = xy[3]
    require_gpu()
    from paper_1709_03187_gb300 import Colony

    col = Colony(xy, **_lbest_kw(50, 2, 5))
    with pytest.raises(AcoError):
        col.build_candidates()


# ------------------------------------------------------------------ tour lengths
@pytest.mark.parametrize("n,count", [(3, 4), (1000, 64), (4097, 9)])
def test_tour_lengths_bit_exact(n, count):
    xy = aco_synth.clustered(n, 5, 0.1, n)
    col, _ = pair(xy, **_lbest_kw(n, 1, min(4, n - 1)))
    rng = np.random.default_rng(n)
    tours = np.stack([rng.permutation(n) for _ in range(count)]).astype(np.int32)
    got = col.tour_lengths(torch.from_numpy(tours)).cpu().numpy()
    want = oracle.tour_lengths(xy, tours)
    assert np.array_equal(got, want)
    empty = col.tour_lengths(torch.from_numpy(tours[:0]))  # no tours: nothing to do
    assert empty.numel() == 0


# ------------------------------------------------------------------ dense mode (Section 2)
@pytest.mark.parametrize("n,m,iters,alpha,beta", [(100, 100, 12, 1.0, 2.0), (37, 9, 20, 2.0, 3.0),
                                                  (3, 2, 5, 1.0, 2.0), (200, 40, 4, 1.0, 5.0)])
def test_dense_iterations_bit_exact(n, m, iters, alpha, beta):
    xy = aco_synth.uniform(n, 1)
    kw = dict(mode=DENSE, n=n, m=m, k=0, alpha=alpha, beta=beta, rho=0.5, tau0=1.0, seed=1)
    col, ref = pair(xy, **kw)
    col.build_candidates()
    for it in range(iters):
        tours, lens = col.construct(it, return_tours=True, return_lengths=True)
        ref.construct(it)
        d = first_divergence(tours.cpu().numpy(), ref.newtours)
        assert d is None, f"iteration {it}: first differing (ant, position) {d}"
        assert np.array_equal(lens.cpu().numpy(), ref.newlen)
        col.update()
        ref.update()
        _, _, tau = col.state()
        assert np.array_equal(tau.cpu().numpy(), ref.tau), f"tau differs after iteration {it}"


def test_dense_probabilities_within_1e5():
    n = 100
    xy = aco_synth.uniform(n, 1)
    kw = dict(mode=DENSE, n=n, m=10, k=0, alpha=1.0, beta=2.0, rho=0.5, tau0=1.0, seed=1)
    col, ref = pair(xy, **kw)
    col.build_candidates()
    for it in range(3):
        col.iterate(it)
        ref.iterate(it)
    rng = np.random.default_rng(0)
    for _ in range(20):
        vis = rng.random(n) < rng.random()
        i = int(rng.integers(n))
        vis[i] = True
        if vis.all():
            continue
        p_gpu, _ = col.step_probs(i, vis)
        p_ref, _ = ref.step_probs(i, vis.astype(np.uint8))
        assert np.max(np.abs(p_gpu.cpu().numpy().astype(np.float64) - p_ref)) < 1e-5


# ------------------------------------------------------------------ PartialACO (Section 3)
@pytest.mark.parametrize("n,m,k,f,iters,p_partial,fallback", [
    (500, 32, 10, 0.3, 25, 1.0, 0),
    (300, 16, 6, 1.0, 20, 1.0, 0),
    (400, 24, 8, 0.2, 15, 0.7, 0),
    (257, 8, 5, 0.5, 10, 0.8, 1),
    (3, 4, 2, 1.0, 6, 1.0, 0),
    (33, 5, 32, 0.5, 8, 1.0, 0),
    (1000, 64, 16, 0.01, 10, 1.0, 0),
    (40, 1, 6, 0.5, 8, 1.0, 0),      # a single ant
    (60, 6, 1, 0.5, 6, 1.0, 0),      # one candidate: nearly every step is an exhausted step
    (90, 5, 2, 1.0, 6, 0.5, 1),      # two candidates, the Eq. 1 wheel over all unvisited
    (600, 1032, 8, 0.3, 4, 1.0, 0),  # m > 1024: rebuild weights from shared memory, rank rows in blocks
    (300, 1030, 6, 0.5, 3, 1.0, 0),  # m > 1024 and not a multiple of 8: the scalar rank-row paths
    (12000, 8, 16, 0.05, 3, 1.0, 0),  # above 8,192 cities: initial tours read the 128-nearest lists
    (10000, 6, 20, 0.05, 2, 1.0, 0),
    (700, 24, 24, 0.3, 8, 1.0, 0),   # the widest stage (k = 24 rows of 24 entries)
    (500, 16, 18, 0.4, 8, 0.8, 0),   # k = 18 on the wide stage, full tours mid-run
    (400, 12, 21, 0.3, 6, 1.0, 0),   # odd k above 16: rows read from global memory
])
def test_partialaco_iterations_bit_exact(n, m, k, f, iters, p_partial, fallback):
    xy = aco_synth.clustered(n, max(1, n // 50), 0.02, n + m)
    col, ref = pair(xy, **_lbest_kw(n, m, k, f=f, seed=n * 7 + 1, p_partial=p_partial, fallback=fallback))
    col.build_candidates()
    for it in range(iters):
        tours, lens = col.construct(it, return_tours=True, return_lengths=True)
        ref.construct(it)
        d = first_divergence(tours.cpu().numpy(), ref.newtours)
        assert d is None, f"iteration {it}: first differing (ant, position) {d}"
        assert np.array_equal(lens.cpu().numpy(), ref.newlen)
        col.update()
        ref.update()
        lb, cl, _ = col.state()
        assert np.array_equal(lb.cpu().numpy(), ref.lbest)
        assert np.array_equal(cl.cpu().numpy(), ref.clen)
    st = col.stats()
    assert st["gbest"] == ref.clen.min()
    c = ref.counters()
    assert st["decisions"] == c["decisions"]
    assert st["fallbacks"] == c["fallbacks"]


def test_candidate_probabilities_within_1e5():
    n, m, k = 800, 32, 16
    xy = aco_synth.clustered(n, 8, 0.03, 5)
    col, ref = pair(xy, **_lbest_kw(n, m, k, f=0.2))
    col.build_candidates()
    for it in range(6):
        col.iterate(it)
        ref.iterate(it)
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(40):
        vis = rng.random(n) < 0.5
        i = int(rng.integers(n))
        p_gpu, ex_gpu = col.step_probs(i, vis)
        p_ref, ex_ref = ref.step_probs(i, vis.astype(np.uint8))
        assert ex_gpu == ex_ref
        if not ex_ref:
            worst = max(worst, float(np.max(np.abs(p_gpu.cpu().numpy().astype(np.float64) - p_ref))))
    assert worst < 1e-5


def test_checkpoint_resume_reproduces_run():
    n, m, k = 400, 16, 8
    xy = aco_synth.uniform(n, 9)
    kw = _lbest_kw(n, m, k, f=0.25, seed=5)
    require_gpu()
    from paper_1709_03187_gb300 import Colony

    a = Colony(xy, **kw)
    a.build_candidates()
    for it in range(5):
        a.iterate(it)
    lb, cl, _ = a.state()
    b = Colony(xy, **kw)
    b.build_candidates()
    b.set_state(lbest=lb)
    _, cl_b, _ = b.state()
    assert torch.equal(cl, cl_b)
    for it in range(5, 12):
        a.iterate(it)
        b.iterate(it)
    assert torch.equal(a.state()[0], b.state()[0])


def test_call_order_and_arguments():
    from paper_1709_03187_gb300 import AcoError, Colony

    require_gpu()
    xy = aco_synth.uniform(20, 2)
    with pytest.raises(AcoError):
        Colony(xy, **_lbest_kw(20, 4, 20))  # k > n - 1
    with pytest.raises(AcoError):
        Colony(xy[:2].copy(), **_lbest_kw(2, 4, 1))  # n < 3
    col = Colony(xy, **_lbest_kw(20, 4, 5))
    with pytest.raises(AcoError):
        col.construct(0)  # before build_candidates
    col.build_candidates()
    with pytest.raises(AcoError):
        col.update()  # before construct
    bad = np.zeros((1, 20), np.int32)
    bad[0, 3] = 99
    col.tour_lengths(torch.from_numpy(bad))  # out-of-range index: skipped, flagged on the device
    with pytest.raises(AcoError):
        col.stats()


def test_lattice_initial_tours_above_the_far_list_size():
    """A 100 x 100 lattice (exact distance ties everywhere) above 8,192 cities: the initial tours,
    whose exhausted steps read the 128-nearest lists ordered by (d^2, index), and one PartialACO
    iteration, bit for bit against the oracle."""
    g = np.arange(100, dtype=np.float64)
    xy = np.ascontiguousarray(np.stack(np.meshgrid(g, g), -1).reshape(-1, 2))
    n = xy.shape[0]
    col, ref = pair(xy, **_lbest_kw(n, 4, 8, f=0.05, seed=5))
    col.build_candidates()
    for it in range(2):
        tours, _ = col.construct(it, return_tours=True, return_lengths=True)
        ref.construct(it)
        d = first_divergence(tours.cpu().numpy(), ref.newtours)
        assert d is None, f"iteration {it}: first differing (ant, position) {d}"
        col.update()
        ref.update()
