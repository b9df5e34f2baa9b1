"""Distribution of the pair tiles over ranks (Section III-D).

The paper gives process i of p the tile ids
    [i * ceil(T/p), (i+1) * ceil(T/p))       with T = m(m+1)/2 tiles,
and has every process run the same tiled computation on its own range; the
ranges are disjoint and no data moves between processes while they compute.
The last ranges can run past T, so they are clamped to T here.

On GB300 one rank drives one GPU: ``allpairs_sharded`` computes the rank's
range into that rank's packed output through pcc_allpairs_upper (entries
outside the range are left untouched), so a caller that wants the whole
triangle in one place gathers the ranks' outputs afterwards (or writes them
to disjoint files); nothing in the computation needs a collective.
"""
from __future__ import annotations


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
