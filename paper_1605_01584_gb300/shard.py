"""Distribution of the pair tiles over ranks (Section III-D).

The paper gives process i of p the tile ids
    [i * ceil(T/p), (i+1) * ceil(T/p))       with T = m(m+1)/2 tiles,
and has every process run the same tiled computation on its own range; the
ranges are disjoint and no data moves between processes while they compute.
The last ranges can run past T, so they are clamped to T here.

On GB300 one rank drives one GPU: ``allpairs_sharded`` computes the rank's
range into that rank's packed output through pcc_allpairs_upper (entries
outside the range are left untouched); nothing in the computation needs a
collective.  A tile range covers a known set of packed runs (each row of a
tile is one contiguous run of the packed triangle, ``tile_runs``), so the
whole triangle is assembled afterwards on the host: ``gather_upper``
collects every rank's runs on one rank over the host process group, and
``write_upper_shard`` has every rank write its own runs into one shared
file (disjoint byte ranges, no communication at all).
"""
from __future__ import annotations

import numpy as np


def tile_range(rank: int, world: int, total: int):
    """[begin, end) of the tile ids of `rank` among `world` ranks."""
    if world < 1 or not (0 <= rank < world) or total < 0:
        raise ValueError("bad rank/world/total")
    per = -(-total // world)  # ceil(T / p)
    begin = min(rank * per, total)
    end = min((rank + 1) * per, total)
    return begin, end


def allpairs_sharded(Z, R, rank: int, world: int, stream=None):
    """Compute this rank's tiles of Z's schedule into R (device, packed)."""
    from . import pcc_allpairs_upper
    b, e = tile_range(rank, world, Z.num_tiles())
    if e > b:
        pcc_allpairs_upper(Z, R, b, e, stream=stream)
    return b, e


def tile_runs(n: int, prec, tile_begin: int, tile_end: int):
    """Packed runs written by tiles [tile_begin, tile_end) of the schedule
    of a Z with n rows in form prec: (starts, lengths) int64 arrays, one run
    per row of each tile (J(i, j0) .. J(i, j1 - 1) for the tile's columns
    j0 <= j < j1 with j > i), in tile order."""
    from . import pcc_schedule_tile_rect
    starts, lens = [], []
    for t in range(tile_begin, tile_end):
        r0, r1, c0, c1 = pcc_schedule_tile_rect(n, prec, t)
        i = np.arange(r0, r1, dtype=np.int64)
        j0 = np.maximum(c0, i + 1)
        ln = c1 - j0
        keep = ln > 0
        i, j0, ln = i[keep], j0[keep], ln[keep]
        starts.append(i * (2 * n - i - 1) // 2 + (j0 - i - 1))
        lens.append(ln)
    if not starts:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(starts), np.concatenate(lens)


def _run_index(starts, lens):
    """Flat packed indices of the runs, in run order."""
    total = int(lens.sum())
    if total == 0:
        return np.zeros(0, np.int64)
    first = np.repeat(starts - np.concatenate(([0], np.cumsum(lens)[:-1])),
                      lens)
    return first + np.arange(total, dtype=np.int64)


def _host_array(R):
    if hasattr(R, "detach"):  # a torch tensor (host or device)
        return R.detach().cpu().numpy()
    return np.asarray(R)


def rank_values(R_local, n: int, prec, rank: int, world: int):
    """This rank's entries of its packed output R_local (host or device,
    n(n-1)/2 elements), in the order of tile_runs over its tile range."""
    b, e = tile_range(rank, world, _num_tiles(n, prec))
    return _host_array(R_local)[_run_index(*tile_runs(n, prec, b, e))]


def _num_tiles(n, prec):
    from . import pcc_schedule_num_tiles
    T = pcc_schedule_num_tiles(n, prec)
    if T < 0:
        raise ValueError("bad n or prec")
    return T


def gather_upper(R_local, n: int, prec, rank: int, world: int, dist=None,
                 dst: int = 0):
    """Assemble the whole packed triangle on rank `dst` from every rank's
    own tile range (Section III-D): each rank sends only the runs its range
    wrote, over the host process group `dist` (torch.distributed with CPU
    tensors; gloo, or any backend that gathers host tensors); rank dst
    places them by the same run lists, which every rank can compute without
    communication.  Returns the host triangle on dst, None elsewhere.  With
    dist None (one process) world must be 1."""
    import torch
    vals = rank_values(R_local, n, prec, rank, world)
    npairs = n * (n - 1) // 2
    if dist is None:
        if world != 1:
            raise ValueError("several ranks need a process group")
        out = np.empty(npairs, dtype=vals.dtype)
        out[_run_index(*tile_runs(n, prec, 0, _num_tiles(n, prec)))] = vals
        return out
    T = _num_tiles(n, prec)
    sizes = [int(_run_index(*tile_runs(n, prec, *tile_range(r, world, T)))
                 .size) for r in range(world)]
    mx = max(sizes + [1])
    pad = torch.zeros(mx, dtype=torch.from_numpy(vals[:0]).dtype)
    pad[:vals.size] = torch.from_numpy(vals)
    bufs = [torch.empty_like(pad) for _ in range(world)] if rank == dst \
        else None
    dist.gather(pad, gather_list=bufs, dst=dst)
    if rank != dst:
        return None
    out = np.empty(npairs, dtype=vals.dtype)
    for r in range(world):
        idx = _run_index(*tile_runs(n, prec, *tile_range(r, world, T)))
        out[idx] = bufs[r].numpy()[:sizes[r]]
    return out


def write_upper_shard(path: str, R_local, n: int, prec, rank: int,
                      world: int):
    """Write this rank's runs of the packed triangle into the file `path`
    (n(n-1)/2 elements of R_local's type, raw, row i's pairs contiguous);
    the ranks' runs are disjoint, so every rank writes its own without
    coordination.  The file is created (or extended) to its full size by
    whichever rank opens it first."""
    import os
    vals = rank_values(R_local, n, prec, rank, world)
    b, e = tile_range(rank, world, _num_tiles(n, prec))
    starts, lens = tile_runs(n, prec, b, e)
    isz = vals.dtype.itemsize
    size = n * (n - 1) // 2 * isz
    fd = os.open(path, os.O_RDWR | os.O_CREAT, 0o644)
    try:
        if os.fstat(fd).st_size < size:
            os.ftruncate(fd, size)
        off = 0
        for st, ln in zip(starts.tolist(), lens.tolist()):
            os.pwrite(fd, vals[off:off + ln].tobytes(), st * isz)
            off += ln
    finally:
        os.close(fd)
