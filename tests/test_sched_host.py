"""The tensor-core pair schedule on the host: the banded super-tile order of
pcc_sched.h, compiled with g++ (the header is host and device code).

For each band of G super-tile rows, the order is its g x g diagonal block
numbered by Eq. (9)-(10), then the block to its right column by column
(Eq. (7)-(8) with rows and columns exchanged).  The expected sequence is
built here from that definition alone; the walk must reproduce it exactly,
cover every super-tile of the m x m upper triangle once, and give the same
tiles when a persistent grid of W workers strides over it (each worker's
cursor jumping over whole bands)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1605_01584_gb300", "csrc", "pcc_sched.h")

PROG = r"""
#include <stdio.h>
#include <stdlib.h>
#include "pcc_sched.h"
// argv: m G W.  Prints, for each worker w < W, the tiles w, w + W, ...
// as "t yt xt" lines, each worker with its own cursor.
int main(int argc, char** argv) {
  long long m = atoll(argv[1]), G = atoll(argv[2]), W = atoll(argv[3]);
  long long total = 0;
  for (long long b = 0; b * G < m; ++b) total += pcc::band_tiles(m, G, b);
  printf("%lld\n", total);
  for (long long w = 0; w < W; ++w) {
    pcc::BandCursor c;
    pcc::band_cursor_init(&c, m, G);
    for (long long t = w; t < total; t += W) {
      int64_t y, x;
      pcc::band_tile_coords(&c, m, G, t, &y, &x);
      printf("%lld %lld %lld\n", t, (long long)y, (long long)x);
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def walker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("sched")
    src = d / "walk.cc"
    src.write_text(PROG)
    exe = d / "walk"
    subprocess.run([gxx, "-O1", "-std=c++17", "-I",
                    os.path.dirname(HDR), str(src), "-o", str(exe)],
                   check=True)

    def run(m, G, W=1):
        out = subprocess.run([str(exe), str(m), str(G), str(W)],
                             capture_output=True, text=True,
                             check=True).stdout.split("\n")
        total = int(out[0])
        rows = np.array([list(map(int, s.split())) for s in out[1:] if s],
                        dtype=np.int64).reshape(-1, 3)
        return total, rows
    return run


def expected_order(m, G):
    seq = []
    for r0 in range(0, m, G):
        g = min(G, m - r0)
        for y in range(g):                 # Eq. (9)-(10) on the g x g block
            for x in range(y, g):
                seq.append((r0 + y, r0 + x))
        for x in range(r0 + g, m):         # then column by column
            for y in range(r0, r0 + g):
                seq.append((y, x))
    return seq


@pytest.mark.parametrize("m,G", [(1, 32), (2, 1), (5, 2), (7, 3), (32, 32),
                                 (33, 32), (64, 32), (100, 8), (257, 32),
                                 (300, 7)])
def test_band_order_is_the_definition(walker, m, G):
    total, rows = walker(m, G)
    assert total == m * (m + 1) // 2
    assert np.array_equal(rows[:, 0], np.arange(total))
    got = [tuple(r) for r in rows[:, 1:].tolist()]
    assert got == expected_order(m, G)
    assert len(set(got)) == total          # every super-tile once
    assert all(0 <= y <= x < m for y, x in got)


@pytest.mark.parametrize("m,G,W", [(64, 32, 76), (257, 32, 76), (300, 7, 5),
                                   (33, 2, 1000)])
def test_strided_workers_cover_every_tile_once(walker, m, G, W):
    total, rows = walker(m, G, W)
    assert rows.shape[0] == total
    order = np.argsort(rows[:, 0], kind="stable")
    assert np.array_equal(rows[order, 0], np.arange(total))
    got = [tuple(r) for r in rows[order, 1:].tolist()]
    assert got == expected_order(m, G)
