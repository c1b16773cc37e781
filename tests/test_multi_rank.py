"""The multi-GPU form is replicas only: each rank solves its own realisations and the bench
combines the ranks' numbers (time = max over ranks, eigenpairs and launches = sum).  Covered
here on the CPU with world size 2 over gloo (no GPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times, counts = bench.combine_ranks((1.5 + rank, 2.0 - rank), (100 + rank, 7 * (rank + 1)), world, "cpu")
        out[rank] = (times, counts)
    finally:
        dist.destroy_process_group()


def test_combine_two_ranks_over_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        times, counts = out[r]
        assert times == [2.5, 2.0]                 # max over ranks of each time
        assert counts == [201, 21]                 # sum over ranks of each count


def test_single_rank_combine_is_identity():
    assert bench.combine_ranks((3.0, 4.0), (5, 6), 1, "cpu") == ([3.0, 4.0], [5, 6])


@pytest.mark.parametrize("world", [1, 2, 3])
def test_realisations_disjoint_per_step(world):
    for i in range(6):
        rs = [bench.realisation(r, world, i) for r in range(world)]
        assert len(set(rs)) == len(rs)                     # no two ranks solve the same realisation
        assert all(0 <= r < len(bench.W_LIST) for r in rs)
