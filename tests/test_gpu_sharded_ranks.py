"""One colony split by ants over two processes on the one GPU, each a ShardedColony rank exchanging
its commit records over torch.distributed (gloo: the records go through host memory), equals a
single colony bit for bit.  No kernel of one process waits on the other: the exchange is host-side
collectives between launches.  This runs the package's multi-rank path end to end."""
import os
import socket

import numpy as np
import pytest

import aco_synth
from tests.gpu_common import require_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, M, K, ITERS = 3000, 64, 16, 6


def _params():
    return dict(mode=1, n=N, m=M, k=K, alpha=1.0, beta=2.0, tau0=1.0, max_mod_frac=0.2, p_partial=1.0, seed=77)


def _xy():
    return aco_synth.clustered(N, 15, 0.02, 77)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1709_03187_gb300 import ShardedColony

        col = ShardedColony(_xy(), rank=rank, world=world, **_params())
        col.build_candidates()
        hist = []
        for it in range(ITERS):
            col.iterate(it)
            lb, cl, _ = col.state()
            hist.append((lb.cpu().numpy(), cl.cpu().numpy()))
        q.put((rank, hist, col.stats()["decisions"]))
        col.close()
    finally:
        dist.destroy_process_group()


def test_two_processes_equal_the_single_colony():
    require_gpu()
    import torch.multiprocessing as mp

    from paper_1709_03187_gb300 import Colony

    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=600) for _ in range(world)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    single = Colony(_xy(), **_params())
    single.build_candidates()
    for it in range(ITERS):
        single.iterate(it)
        lb, cl, _ = single.state()
        for rank, hist, _ in out:
            assert np.array_equal(hist[it][0], lb.cpu().numpy()), f"rank {rank}, iteration {it}: l_best"
            assert np.array_equal(hist[it][1], cl.cpu().numpy()), f"rank {rank}, iteration {it}: lengths"
    assert sum(o[2] for o in out) == single.stats()["decisions"]
    single.close()
