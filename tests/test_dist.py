"""Data-parallel host logic on CPU with world_size-2 gloo ranks (no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2503_21935_gb300.dist import event_range, split_range


def test_ranges_partition_events():
    for world in (1, 2, 3, 8):
        got = [split_range(r, world, 1000) for r in range(world)]
        assert sum(n for _, n in got) == 1000
        assert all(got[i][0] + got[i][1] == got[i + 1][0] for i in range(world - 1))
        w = [event_range(r, world, 64) for r in range(world)]
        assert [f for f, _ in w] == [64 * r for r in range(world)]
    with pytest.raises(ValueError):
        event_range(2, 2, 10)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from phasespace import WORKLOADS, make_inputs
    from paper_2503_21935_gb300.dist import event_range, max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, n = event_range(rank, world, 16)
    mom, a, rh, rc = make_inputs(WORKLOADS["ggttg"], n, first=first)
    # each rank's shard equals the matching slice of a single-process generation
    full = make_inputs(WORKLOADS["ggttg"], 16 * world)
    ok = all(np.array_equal(x, y[first:first + n]) for x, y in zip((mom, a, rh, rc), full))
    t = max_over_ranks(1.0 + rank)
    out[rank] = (ok, t, float(mom[:, 2, 0].sum()))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert out[0][0] and out[1][0]
    assert out[0][1] == out[1][1] == 2.0            # max over ranks seen by every rank
    assert out[0][2] != out[1][2]                    # different events on different ranks
