"""Host logic of the N > 1 bench paths on CPU ranks (gloo, world size 2): the
size-balanced share-out of independent slices (no collective on the data
path) and the max-over-ranks timing that every rank agrees on."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

import bench                               # noqa: E402
from workloads import batched_slices      # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_every_slice_once_and_balances():
    sizes = [d["n"] ** 2 for d in batched_slices(64, 2026)]
    for world in (1, 2, 3, 8):
        parts = bench.partition_slices(sizes, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(64))
        loads = [sum(sizes[k] for k in p) for p in parts]
        # greedy largest-first: no rank exceeds the mean by more than the largest slice
        assert max(loads) - sum(loads) / world <= max(sizes)
    assert bench.partition_slices([5, 1, 1, 1], 2) == [[0], [1, 2, 3]]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        sizes = [d["n"] ** 2 for d in batched_slices(64, 2026)]
        mine = bench.partition_slices(sizes, world)[rank]
        got = [None] * world
        dist.all_gather_object(got, mine)
        out[rank] = (ms, got)
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_agree():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert [res[r][0] for r in range(world)] == [15.0, 15.0]      # the slowest rank's time
    shares = res[0][1]
    assert shares == res[1][1]
    assert sorted(k for p in shares for k in p) == list(range(64))
    assert not set(shares[0]) & set(shares[1])
