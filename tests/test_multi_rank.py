"""The N > 1 path of the benchmark on CPU: world size 2 over gloo (127.0.0.1).

The ranks run one colony split by ants (its exchange is tested in test_multi_rank_sharded.py);
here: the whole-job aggregation (the slowest rank's time, the sum of the units every rank
processed) and the reference arm, which runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        t, u = bench.aggregate_over_ranks(1.0 + 0.5 * rank, 10.0 * (rank + 1), world, "cpu")
        ranks = [None] * world
        dist.all_gather_object(ranks, rank)
        ran_reference = []

        class _Args:
            workload = "dense100"

        # rank != 0 returns before touching the oracle or any work
        if rank != 0:
            ran_reference.append(bench.run_reference(_Args()) is None)
        q.put((rank, t, u, ranks, ran_reference))
    finally:
        dist.destroy_process_group()


def test_two_ranks_aggregate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u, ranks, ran in out:
        assert t == 1.5 and u == 30.0  # slowest rank's time; units of both ranks
        assert ranks == [0, 1]
        if rank == 1:
            assert ran == [True]


def test_single_rank_is_the_identity():
    import bench

    assert bench.aggregate_over_ranks(2.5, 7, 1) == (2.5, 7.0)
