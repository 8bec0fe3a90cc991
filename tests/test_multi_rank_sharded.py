"""One colony split by ants over two ranks (gloo, 127.0.0.1) equals the single colony, on CPU.

Each rank runs the oracle on its half of the ants, exports the commits of its ants that improved
(the library's record format), and the ranks exchange them with the package's
``exchange_records`` (the same host code the GPU ranks use, here on host tensors over gloo).
Every rank then applies every commit and updates.  Ants read the pheromone synchronously
(Section 3), so after every iteration both ranks hold the single colony's l_best bit for bit, and
so do their new tours and counters summed over the ranks.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

N, M, K, ITERS = 400, 30, 8, 7


def _params(p_partial):
    return dict(mode=1, n=N, m=M, k=K, alpha=1.0, beta=2.0, tau0=1.0, max_mod_frac=0.25, p_partial=p_partial,
                seed=31, fallback=0)


def _xy():
    import aco_synth

    return aco_synth.clustered(N, 6, 0.03, 31)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, p_partial, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1709_03187_gb300.sharded import ant_range, exchange_records

        a0, a1 = ant_range(M, rank, world)
        ref = oracle.Oracle(_xy(), **_params(p_partial))
        history = []
        for it in range(ITERS):
            ref.construct(it, ants=np.arange(a0, a1, dtype=np.int32))
            local = ref.export_commits(a0, a1)
            recs = exchange_records(torch.from_numpy(local), local.size, world=world)
            ref.import_commits([r.numpy() for r in recs], a0, a1)
            ref.update()
            history.append((ref.lbest.copy(), ref.clen.copy()))
        q.put((rank, history, ref.counters()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("p_partial", [1.0, 0.6])
def test_two_ranks_split_by_ants_equal_the_single_colony(p_partial):
    import oracle

    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, p_partial, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=300) for _ in range(world)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    single = oracle.Oracle(_xy(), **_params(p_partial))
    for it in range(ITERS):
        single.iterate(it)
        for rank, history, _ in out:
            lb, cl = history[it]
            assert np.array_equal(lb, single.lbest), f"rank {rank}, iteration {it}"
            assert np.array_equal(cl, single.clen), f"rank {rank}, iteration {it}"
    c = single.counters()
    assert sum(o[2]["decisions"] for o in out) == c["decisions"]
    assert sum(o[2]["fallbacks"] for o in out) == c["fallbacks"]


def test_exchange_pads_rows_to_an_even_stride():
    """One rank: the gathered buffer keeps 8-byte alignment (even stride) and the words."""
    from paper_1709_03187_gb300.sharded import ant_range

    assert [ant_range(10, r, 3) for r in range(3)] == [(0, 3), (3, 6), (6, 10)]
    assert ant_range(7, 0, 1) == (0, 7)
