"""ShardedColony: one colony whose ants are split over the ranks of a torch.distributed group.

Section 3's colony takes its pheromone from every ant's l_best and, read synchronously, every ant
of an iteration sees the same pheromone: the ants can be built on different GPUs.  Each rank keeps
the whole colony state, builds its share of the ants, and one exchange per iteration gives every
rank every commit (the records of ``aco_export_commits``).  Each rank then applies them and runs
the same update, so every rank holds the single colony's state bit for bit.  The exchange is one
all-gather of the record counts and one all-gather of the record buffers (NCCL between GPUs; any
torch.distributed backend works, e.g. gloo for host tensors).
"""
from __future__ import annotations

import torch

from . import _ffi
from .colony import Colony


def ant_range(m: int, rank: int, world: int):
    """The ants of `rank`: [rank m / world, (rank + 1) m / world)."""
    return rank * m // world, (rank + 1) * m // world


def exchange_records(local: torch.Tensor, words: int, group=None, world: int | None = None) -> torch.Tensor:
    """All-gather of variable-length int32 record buffers: `local[:words]` of every rank, padded to
    the longest, as a (world, stride) tensor on local's device (stride even, so every row stays
    8-byte aligned).  Collective: every rank of the group calls it."""
    import torch.distributed as dist

    world = world or dist.get_world_size(group)
    # a backend without device collectives (gloo) exchanges through host memory
    dev = local.device
    via_host = dev.type == "cuda" and dist.get_backend(group) == "gloo"
    cdev = torch.device("cpu") if via_host else dev
    size = torch.tensor([words], dtype=torch.int64, device=cdev)
    sizes = [torch.zeros_like(size) for _ in range(world)]
    dist.all_gather(sizes, size, group=group)
    stride = max(int(s.item()) for s in sizes)
    stride += stride & 1
    send = torch.zeros(stride, dtype=torch.int32, device=cdev)
    send[:words] = local[:words].to(cdev)
    recv = [torch.empty(stride, dtype=torch.int32, device=cdev) for _ in range(world)]
    dist.all_gather(recv, send, group=group)
    return torch.stack(recv).to(dev)


class ShardedColony:
    """This rank's part of one colony split by ants over `world` ranks (parameters as Colony).

    Every rank passes the same coordinates and parameters.  ``iterate`` is collective."""

    def __init__(self, xy, *, rank: int, world: int, group=None, stream: torch.cuda.Stream | None = None, **params):
        self.rank, self.world, self.group = rank, world, group
        self.col = Colony(xy, stream=stream, **params)
        self.n, self.m = self.col.n, self.col.m
        self.ant0, self.ant1 = ant_range(self.m, rank, world)
        _ffi.aco_set_ant_range(self.col.handle, self.ant0, self.ant1)
        # enough for every own ant committing a full tour (the first iteration)
        self.cap = (self.ant1 - self.ant0) * (12 + self.n) + 4
        self.buf = torch.empty(self.cap, dtype=torch.int32, device=self.col.device) if world > 1 else None
        self.exchanged_words = 0

    @property
    def handle(self):
        return self.col.handle

    def build_candidates(self, return_lists: bool = False):
        return self.col.build_candidates(return_lists)

    def construct(self, iteration: int):
        """This rank's ants build their tours (enqueued)."""
        self.col.construct(iteration)

    def exchange(self):
        """Every rank's commits into this rank's instance (collective)."""
        if self.world == 1:
            return
        h = self.col.handle
        words = _ffi.aco_export_commits(h, self.buf, self.cap)
        with torch.cuda.stream(self.col.stream) if self.col.stream is not None else _null():
            recs = exchange_records(self.buf, words, self.group, self.world)
        _ffi.aco_import_commits(h, recs, self.world, recs.shape[1])
        self.exchanged_words = int(recs.shape[0] * recs.shape[1])
        self._recs = recs  # kept alive until the update has read it

    def update(self):
        self.col.update()
        self._recs = None

    def iterate(self, iteration: int):
        self.construct(iteration)
        self.exchange()
        self.update()

    def state(self):
        return self.col.state()

    def stats(self) -> dict:
        return self.col.stats()

    def close(self):
        self.col.close()


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False
