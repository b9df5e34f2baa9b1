"""The multi-rank path on CPU: world-size-2 gloo process group.

Each rank takes its tile range (Section III-D, clamped), maps every tile to
its pairs with the library's host twin of the Eq. (17)-(19) tile bijection
(pcc_tile_coords, the FP32 path's tile order with 128-wide tiles), computes
those pairs with the oracle, and the ranks all-gather (pair index, r)
lists: the union must be the whole packed triangle, exactly once, equal to
the oracle's one-process result.  No GPU is involved."""
import os
import socket

import numpy as np
import pytest

from paper_1605_01584_gb300 import shard


def test_tile_range_partitions():
    for total in (0, 1, 5, 131, 136, 131328):
        for world in (1, 2, 3, 7, 16):
            got = [shard.tile_range(r, world, total) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == total
            for (a, b), (c, d) in zip(got, got[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in got]
            assert max(sizes) <= -(-total // world)
    with pytest.raises(ValueError):
        shard.tile_range(2, 2, 10)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, n, l, out_q):
    import torch
    import torch.distributed as dist

    import oracle
    import paper_1605_01584_gb300 as pcc
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pcc.load()
        X = synth.counts_log(n, l, 13)
        t = 128
        m = -(-n // t)
        b, e = shard.tile_range(rank, world, m * (m + 1) // 2)
        I, J = [], []
        for tid in range(b, e):
            yt, xt = pcc.pcc_tile_coords(m, tid)
            for i in range(yt * t, min(n, (yt + 1) * t)):
                for j in range(max(i + 1, xt * t), min(n, (xt + 1) * t)):
                    I.append(i)
                    J.append(j)
        I = np.array(I, dtype=np.int64)
        J = np.array(J, dtype=np.int64)
        r = oracle.pcc_pairs(X, I, J)
        idx = I * (2 * n - I - 1) // 2 + (J - I - 1)
        mine = torch.from_numpy(np.stack([idx.astype(np.float64), r], 1))
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([mine.shape[0]]))
        mx = int(max(s.item() for s in sizes))
        pad = torch.full((mx, 2), -1.0, dtype=torch.float64)
        pad[:mine.shape[0]] = mine
        got = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(got, pad)
        if rank == 0:
            allv = torch.cat([g[:int(s.item())] for g, s in zip(got, sizes)])
            out_q.put(allv.numpy())
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_union_is_the_triangle():
    import multiprocessing as mp

    import oracle
    import synth
    n, l = 300, 24
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, n, l, q))
             for r in range(2)]
    for p in procs:
        p.start()
    allv = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    idx = allv[:, 0].astype(np.int64)
    npairs = n * (n - 1) // 2
    assert np.array_equal(np.sort(idx), np.arange(npairs))  # exactly once
    want = oracle.pcc_upper(synth.counts_log(n, l, 13))
    got = np.empty(npairs)
    got[idx] = allv[:, 1]
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.array_equal(got[ok], want[ok])


def _bench_rank_main(rank, world, port, out_q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank's step time differs; every rank must see the slowest
        got = bench.max_over_ranks(4.5 + 1.25 * rank, dist)
        dist.barrier()
        out_q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_bench_times_are_the_max_over_ranks():
    """bench.py's multi-rank timing: the step time every rank reports is
    the slowest rank's (the whole-job value divides all ranks' work by it)."""
    import multiprocessing as mp

    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_rank_main, args=(r, 2, port, q))
             for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res == {0: 5.75, 1: 5.75}
