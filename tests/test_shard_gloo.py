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


def _tc_rank_main(rank, world, port, n, l, band, path, out_q):
    """One rank of the tensor-core schedule (banded 256 x 256 super-tiles):
    its tile range's pairs, listed by the library's host schedule, computed
    by the oracle into a packed array of its own (sentinel elsewhere), then
    assembled by shard.gather_upper and shard.write_upper_shard."""
    import torch.distributed as dist

    import oracle
    import paper_1605_01584_gb300 as pcc
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pcc.load()
        pcc.pcc_set_tuning(band_rows=band)  # host knob: no device needed
        X = synth.counts_log(n, l, 17)
        T = pcc.pcc_schedule_num_tiles(n, "fp16x3s")
        b, e = shard.tile_range(rank, world, T)
        I, J = [], []
        for t in range(b, e):
            r0, r1, c0, c1 = pcc.pcc_schedule_tile_rect(n, "fp16x3s", t)
            for i in range(r0, r1):
                js = np.arange(max(c0, i + 1), c1)
                I.append(np.full(js.size, i))
                J.append(js)
        I = np.concatenate(I).astype(np.int64)
        J = np.concatenate(J).astype(np.int64)
        R = np.full(n * (n - 1) // 2, 7.0)
        R[I * (2 * n - I - 1) // 2 + (J - I - 1)] = oracle.pcc_pairs(X, I, J)
        whole = shard.gather_upper(R, n, "fp16x3s", rank, world, dist)
        shard.write_upper_shard(path, R, n, "fp16x3s", rank, world)
        dist.barrier()
        if rank == 0:
            out_q.put((T, whole, np.fromfile(path, dtype=np.float64)))
        else:
            assert whole is None
    finally:
        dist.destroy_process_group()


def test_two_rank_gather_through_tensor_core_schedule(tmp_path):
    """Section III-D's ranges over the tensor-core kernels' banded
    super-tile order: the host gather and the shared file each rebuild the
    whole packed triangle, equal to the oracle's one-process result."""
    import multiprocessing as mp

    import oracle
    import synth
    n, l, band = 1300, 20, 2  # 6 x 6 super-tiles in 3 bands, 21 tiles
    path = str(tmp_path / "upper.f64")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_tc_rank_main,
                         args=(r, 2, port, n, l, band, path, q))
             for r in range(2)]
    for p in procs:
        p.start()
    T, whole, filed = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert T == 21
    want = oracle.pcc_upper(synth.counts_log(n, l, 17))
    for got in (whole, filed):
        assert not np.any(got == 7.0)
        assert np.array_equal(np.isnan(got), np.isnan(want))
        ok = ~np.isnan(want)
        assert np.array_equal(got[ok], want[ok])


def test_schedule_rectangles_cover_each_pair_once():
    """The host schedule's tiles cover every pair i < j exactly once, for
    the tensor-core order at several band heights and the CUDA-core
    order."""
    import paper_1605_01584_gb300 as pcc
    pcc.load()
    before = pcc.pcc_get_tuning()
    try:
        for n, prec, band in [(700, "fp16x3s", 1), (1100, "bf16x3", 3),
                              (1100, "auto", 32), (300, "fp32", 32),
                              (200, "fp64", 32)]:
            pcc.pcc_set_tuning(band_rows=band)
            T = pcc.pcc_schedule_num_tiles(n, prec)
            starts, lens = shard.tile_runs(n, prec, 0, T)
            idx = shard._run_index(starts, lens)
            assert np.array_equal(np.sort(idx), np.arange(n * (n - 1) // 2))
            parts = [shard.tile_runs(n, prec, *shard.tile_range(r, 3, T))
                     for r in range(3)]
            cat = np.concatenate([shard._run_index(*p) for p in parts])
            assert np.array_equal(cat, idx)
    finally:
        pcc.pcc_set_tuning(band_rows=before["band_rows"])
