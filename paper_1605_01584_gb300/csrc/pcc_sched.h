// pcc_sched.h -- job/tile numbering of the pair schedule (host and device).
//
// Section III-B/C of LightPCC numbers the cells of the upper triangle of an
// m x m matrix (diagonal included) left to right, top to bottom:
//   J_m(y,x) = F_m(y) + x - y,   F_m(y) = y(2m - y + 1)/2        Eq. (9)-(10)
// and inverts it in closed form:
//   y = ceil(m - 0.5 - sqrt(m^2 + m + 0.25 - 2(J+1))),  x = J + y - F_m(y)
//                                                           Eq. (14)-(15)
// The proof is exact-real.  At the last id of a row the square root is an
// exact half-integer, so a floating-point root that lands one ulp low gives
// y+1; the FP64 value is therefore corrected with exact integer tests
// (F_m(y) <= J < F_m(y+1)), which makes the map exact for any m; below
// m = 2^26 the FP64 estimate is already within one row of the answer.
#pragma once
#include <stdint.h>
#include <math.h>

#if defined(__CUDACC__)
#define PCC_HD __host__ __device__ __forceinline__
#else
#define PCC_HD static inline
#endif

namespace pcc {

// F_m(y), Eq. (10)
PCC_HD int64_t tri_F(int64_t m, int64_t y) { return y * (2 * m - y + 1) / 2; }

// Eq. (14)-(15) in FP64 plus the integer correction.  0 <= J < m(m+1)/2.
PCC_HD void tri_coords(int64_t m, int64_t J, int64_t* y, int64_t* x) {
  double md = (double)m;
  double rad = md * md + md + 0.25 - 2.0 * (double)(J + 1);
  if (rad < 0.0) rad = 0.0;
  int64_t yy = (int64_t)ceil(md - 0.5 - sqrt(rad));
  if (yy < 0) yy = 0;
  if (yy > m - 1) yy = m - 1;
  while (yy > 0 && tri_F(m, yy) > J) --yy;
  while (yy + 1 < m && tri_F(m, yy + 1) <= J) ++yy;
  *y = yy;
  *x = J + yy - tri_F(m, yy);
}

// Strict upper triangle (i < j) of n variables = the diagonal-inclusive
// triangle of n-1 shifted one column: J(i,j) = F_{n-1}(i) + (j-1) - i.
PCC_HD int64_t pair_row_base(int64_t n, int64_t i) {
  // J(i,j) = pair_row_base(n,i) + j
  return i * (2 * n - i - 1) / 2 - i - 1;
}

// ---------------------------------------------------------------------
// Tensor-core pair schedule.
//
// Super-tiles of T x T pairs (T = 256) form an m x m tile matrix, m =
// ceil(n/T).  Its upper triangle (diagonal included) is walked in bands of G
// tile rows: band b holds tile rows [bG, bG+g), g = min(G, m - bG); first
// its g x g diagonal block (numbered by Eq. (9)-(10) with m = g), then the
// g x (m - bG - g) block to its right in column-major order (Eq. (7)-(8)
// with the roles of x and y exchanged).  Walking columns inside a band keeps
// the band's g row panels hot in L2 while each column panel is read once
// per band.  Tile t = (band prefix) + position; each tile is split into two
// work units of 128 rows x 256 columns (unit = 2t + half).
// ---------------------------------------------------------------------
constexpr int kTcSuper = 256;
constexpr int kTcRows = 128;

PCC_HD int64_t tc_super_count(int64_t n) { return (n + kTcSuper - 1) / kTcSuper; }

PCC_HD int64_t band_tiles(int64_t m, int64_t G, int64_t b) {
  int64_t r0 = b * G;
  int64_t g = m - r0 < G ? m - r0 : G;
  if (g <= 0) return 0;
  return g * (g + 1) / 2 + g * (m - r0 - g);
}

struct BandCursor {
  int64_t band, start, count;
};

PCC_HD void band_cursor_init(BandCursor* c, int64_t m, int64_t G) {
  c->band = 0;
  c->start = 0;
  c->count = band_tiles(m, G, 0);
}

// Map tile t (monotone non-decreasing across calls on one cursor) to its
// super-tile coordinates (yt <= xt).
PCC_HD void band_tile_coords(BandCursor* c, int64_t m, int64_t G, int64_t t,
                             int64_t* yt, int64_t* xt) {
  while (t >= c->start + c->count && c->count > 0) {
    c->start += c->count;
    c->band += 1;
    c->count = band_tiles(m, G, c->band);
  }
  int64_t r0 = c->band * G;
  int64_t g = m - r0 < G ? m - r0 : G;
  int64_t p = t - c->start;
  int64_t tri = g * (g + 1) / 2;
  if (p < tri) {
    int64_t dy, dx;
    tri_coords(g, p, &dy, &dx);
    *yt = r0 + dy;
    *xt = r0 + dx;
  } else {
    int64_t q = p - tri;
    *xt = r0 + g + q / g;
    *yt = r0 + q % g;
  }
}

}  // namespace pcc
