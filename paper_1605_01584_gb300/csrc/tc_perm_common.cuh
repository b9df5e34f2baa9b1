// tc_perm_common.cuh -- what the two forms of the tensor-core permutation
// test share: the 128 x 128 tile of the triangle, the MMA step, and the
// numbering of tile pairs column by column for CTA pairs.
#pragma once
#include <math.h>
#include <stdint.h>

namespace pcc {

constexpr int kPT = 128;                 // tile side (M of one CTA)
constexpr int kPUK = 16;                 // K of one tcgen05.mma (16-bit)
constexpr int kPEpiWarps = 8;            // epilogue warps per CTA
constexpr int kPAcc = 2 * kPT;           // TMEM columns per accumulator
constexpr int kPMaxResidentK = 256;      // resident A tile up to lpad 256
constexpr int kPSmemBudget = 232448;     // dynamic shared memory per CTA

// PAIR items: the tiles of column x of the triangle taken two by two, rows
// (2r, 2r+1); column x holds floor((x+2)/2) pairs (the last one alone when
// x is even) and Q(x) = floor((x+1)/2) * floor((x+2)/2) pairs come before
// it.  The closed-form estimate is corrected by exact integer tests.
__host__ __device__ __forceinline__ int64_t col_pairs_before(int64_t x) {
  return ((x + 1) / 2) * ((x + 2) / 2);
}

__device__ __forceinline__ void col_pair_coords(int64_t t, int64_t* r,
                                                int64_t* x) {
  int64_t xx = (int64_t)(2.0 * sqrt((double)t));
  if (xx < 0) xx = 0;
  while (xx > 0 && col_pairs_before(xx) > t) --xx;
  while (col_pairs_before(xx + 1) <= t) ++xx;
  *x = xx;
  *r = t - col_pairs_before(xx);
}

}  // namespace pcc
