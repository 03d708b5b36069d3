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


def _collective_worker(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2503_21935_gb300 import dist as D
    from oracle import mlp as ref
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert D.rank_world() == (rank, world)
    # weight statistics of rank-dependent batches of different lengths
    rng = np.random.default_rng(100 + rank)
    w = torch.from_numpy(rng.exponential(size=1000 + 37 * rank))
    stats = D.allreduce_weight_stats(float(w.max()), float(w.sum()), w.numel())
    sums = D.allreduce_sums([float(w.sum()), float((w * w).sum()), w.numel()])
    union = D.gather_samples(w)
    # data-parallel gradient: each rank's half of one batch, the float64 reference network
    prng = np.random.default_rng(5)
    p = prng.normal(scale=0.05, size=ref.WIDTH * ref.K0 + 3 * ref.WIDTH * ref.WIDTH + 5 * ref.WIDTH + 1)
    x = prng.normal(size=(64, ref.NIN))
    t = prng.normal(size=64)
    half = slice(32 * rank, 32 * rank + 32)
    _, g = ref.gradients(p, x[half], t[half])
    gt = torch.from_numpy(g.copy())
    total = D.allreduce_gradients(gt, 32)
    out[rank] = (stats, sums, union.numpy(), gt.numpy(), total)
    dist.destroy_process_group()


def test_two_gloo_ranks_collectives():
    """The collectives of the data-parallel unweighting and training, on two gloo ranks: both ranks
    get the same (max w, sum w, N), the same moments and the same union of calibration weights as a
    single process computes from all the data; the averaged gradient of the two half-batches equals
    the float64 reference gradient of the whole batch."""
    import numpy as np
    from paper_2503_21935_gb300 import dist as D
    from oracle import mlp as ref
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_collective_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn",
                       join=True)
    ws = [np.random.default_rng(100 + r).exponential(size=1000 + 37 * r) for r in range(world)]
    every = np.concatenate(ws)
    s0, s1 = out[0], out[1]
    assert s0[0] == s1[0] and s0[1] == s1[1]
    mx, sw, n = s0[0]
    assert mx == every.max() and n == every.size
    assert sw == ws[0].sum() + ws[1].sum()                 # rank-order sum of the per-rank sums
    assert abs(sw / every.sum() - 1) < 1e-14
    assert s0[1][2] == every.size and abs(s0[1][1] / (every ** 2).sum() - 1) < 1e-14
    assert np.array_equal(s0[2], every) and np.array_equal(s1[2], every)
    prng = np.random.default_rng(5)
    p = prng.normal(scale=0.05, size=ref.WIDTH * ref.K0 + 3 * ref.WIDTH * ref.WIDTH + 5 * ref.WIDTH + 1)
    x = prng.normal(size=(64, ref.NIN))
    t = prng.normal(size=64)
    _, g_full = ref.gradients(p, x, t)
    assert s0[4] == s1[4] == 64
    assert np.array_equal(s0[3], s1[3])                    # replicas apply the same update
    assert np.abs(s0[3] - g_full).max() <= 1e-12 * np.abs(g_full).max()
    # the pure combination the collective performs
    halves = [ref.gradients(p, x[:32], t[:32])[1], ref.gradients(p, x[32:], t[32:])[1]]
    assert np.abs(D.combine_gradients(halves, [32, 32]) - g_full).max() <= 1e-12 * np.abs(g_full).max()
    assert D.combine_weight_stats([(1.0, 2.0, 3), (5.0, 1.0, 1)]) == (5.0, 3.0, 4)
